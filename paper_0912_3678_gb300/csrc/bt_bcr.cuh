// Block cyclic reduction (odd-even reduction), the "cyclic reduction"
// factorization of Sec. 2, with one synchronisation (kernel launch) per
// reduction step.  CTA (or 2-CTA cluster) per row, m >= 8.  Level l holds K
// active block rows (B_q, D_q, C_q, f_q); the rows at odd positions are
// eliminated:
//   alpha_q = -B_{2q} D_{2q-1}^{-1},  gamma_q = -C_{2q} D_{2q+1}^{-1}
//   D'_q = D_{2q} + alpha_q C_{2q-1} + gamma_q B_{2q+1}
//   B'_q = alpha_q B_{2q-1},  C'_q = gamma_q C_{2q+1},  f'_q = f_{2q} + alpha_q f_{2q-1} + gamma_q f_{2q+1}
// and after the single remaining row is solved the odd rows are recovered:
//   x_{2q+1} = D_{2q+1}^{-1} (f_{2q+1} - B_{2q+1} x_{2q} - C_{2q+1} x_{2q+2}).
// Two uses: the reduced system T_p (FP64), and the local factorization of
// partitions of 2^L block rows (the steps below level L, which never
// eliminate a row at a multiple of 2^L, so those rows are the separators and
// what is left after L steps is the reduced system on them).  The local steps
// may compute in FP32 (refined paths): each level then computes in type T,
// reads its matrix in type TI and writes the next level's in type TO.
#pragma once
#include <cooperative_groups.h>

#include "bt_cta.cuh"

namespace bt {

struct BcrArgs {
    long long K;          // active rows of this level
    int nr, level;
    int mode;             // BcrMode: arithmetic and storage types of this level
    const void* B;        // [K][m][m] (type TI)
    const void* D;
    const void* C;
    void* Dinv;           // [K/2] inverses of the odd rows (the single row when K == 1), type T
    void* al;             // [(K+1)/2] alpha of the kept rows, type T
    void* ga;             // [(K+1)/2] gamma of the kept rows, type T
    void* Bn;             // next level [(K+1)/2][m][m], type TO
    void* Dn;
    void* Cn;
    const double* F;      // [K][m][nr]
    double* Fn;           // [(K+1)/2][m][nr]
    double* X;            // [K][m][nr]
    const double* Xn;     // [(K+1)/2][m][nr]
    long long* status;
};

// (T, TI, TO) of a level.
enum BcrMode : int {
    BCR_F64 = 0,          // double, double, double
    BCR_F32_FIRST = 1,    // float, double, float   (first local step)
    BCR_F32 = 2,          // float, float, float    (middle local steps)
    BCR_F32_LAST = 3,     // float, float, double   (last local step: the reduced system is FP64)
    BCR_F32_ONLY = 4      // float, double, double  (a single local step)
};

// double -> float by integer operations (no FP64-pipe conversion): the
// mantissa is truncated to 23 bits (relative error below 2^-23, toward zero),
// magnitudes below the FP32 normal range become signed zero, larger ones and
// non-finite values infinity or NaN.  Used where FP32 copies of FP64 data feed
// an FP32 computation that refinement corrects.
__device__ __forceinline__ float trunc_f32(double v) {
    const unsigned hi = (unsigned)__double2hiint(v), lo = (unsigned)__double2loint(v);
    const unsigned sign = hi & 0x80000000u;
    const int e64 = (int)((hi >> 20) & 0x7ffu);
    const int e = e64 - 1023 + 127;
    if (e <= 0) return __uint_as_float(sign);
    if (e >= 255) {
        const bool nan = (e64 == 0x7ff) && (((hi & 0xfffffu) | lo) != 0u);
        return __uint_as_float(sign | 0x7f800000u | (nan ? 0x400000u : 0u));
    }
    return __uint_as_float(sign | ((unsigned)e << 23) | ((hi & 0xfffffu) << 3) | (lo >> 29));
}
// v = hi + lo: hi = v truncated to FP32, lo = the remaining 29 mantissa
// bits, rounded to FP32.  Integer and FP32 operations only (the FP64 pipe,
// which also executes integer-to-float conversions on this GPU, is not used):
// hi is assembled from the exponent and the top 23 fraction bits; the
// remainder L < 2^29 is converted as L = 64 L1 + L0 with each part read off
// 2^23 + L_i (the magic-number conversion), scaled by the weight of its last
// bit.  Magnitudes outside the FP32 range give hi = 0 (below) or infinity
// (above, also NaN); lo is 0 below 2^-74.
__device__ __forceinline__ float2 split_f64(double v) {
    const unsigned hw = (unsigned)__double2hiint(v), lw = (unsigned)__double2loint(v);
    const unsigned sign = hw & 0x80000000u;
    const unsigned e = (hw >> 20) & 0x7ffu;
    const unsigned mant = __funnelshift_l(lw, hw, 3) & 0x7fffffu;
    unsigned hb = sign | ((e - 896u) << 23) | mant;
    if (e - 897u >= 254u) hb = (e < 897u) ? sign : (sign | 0x7f800000u | (((hw & 0xfffffu) | lw) ? 0x400000u : 0u));
    const unsigned L = lw & 0x1fffffffu;
    const float l1 = __fsub_rn(__uint_as_float(0x4b000000u | (L >> 6)), 8388608.f);
    const float l0 = __fsub_rn(__uint_as_float(0x4b000000u | (L & 63u)), 8388608.f);
    const unsigned se = e - 948u;   // FP32 exponent field of 2^(e - 1075), the weight of bit 0
    float lo = __fmul_rn(fmaf(l1, 64.f, l0), __uint_as_float((se << 23) | sign));
    if (se - 1u >= 254u) lo = 0.f;
    return make_float2(__uint_as_float(hb), lo);
}

template <typename T, typename G>
__device__ __forceinline__ T cvt_in(G v) {
    if constexpr (std::is_same<T, G>::value) return v;
    else if constexpr (std::is_same<T, float>::value) return trunc_f32(v);
    else return (T)v;
}

template <typename T, int M, typename G>
__device__ __forceinline__ void load_any(T* s, const G* g) {
    using S = Cta<T, M>;
    for (int idx = threadIdx.x; idx < M * M; idx += S::NT) s[(idx / M) * S::LD + idx % M] = cvt_in<T>(g[idx]);
}

// The reduced levels are small, so these kernels are built for latency: each
// dot product of length M is split over four partial sums (dependency chains
// of M/4 instead of M), and one launch per level does the whole elimination step.

// acc[q] += sgn * (A B)[r0+q][c] over four partial sums.
template <typename T, int M, bool NEG>
__device__ __forceinline__ void gemm_lat(T (&acc)[M / 8], const T* A, const T* B, int r0, int c) {
    constexpr int LD = M + 1, R = M / 8;
    T p[R][4];
#pragma unroll
    for (int q = 0; q < R; ++q)
#pragma unroll
        for (int u = 0; u < 4; ++u) p[q][u] = T(0);
#pragma unroll
    for (int k = 0; k < M; k += 4) {
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const T b = NEG ? -B[(k + u) * LD + c] : B[(k + u) * LD + c];
#pragma unroll
            for (int q = 0; q < R; ++q) p[q][u] = fmaT<T>(A[(r0 + q) * LD + k + u], b, p[q][u]);
        }
    }
#pragma unroll
    for (int q = 0; q < R; ++q) acc[q] += (p[q][0] + p[q][1]) + (p[q][2] + p[q][3]);
}

// sum_k A[row][k] v[k * nr] over four partial sums (A in shared memory, row-padded).
template <typename T, int M>
__device__ __forceinline__ T dot_lat(const T* Arow, const T* v, int nr) {
    T p0 = T(0), p1 = T(0), p2 = T(0), p3 = T(0);
#pragma unroll
    for (int k = 0; k < M; k += 4) {
        p0 = fmaT<T>(Arow[k], v[k * nr], p0);
        p1 = fmaT<T>(Arow[k + 1], v[(k + 1) * nr], p1);
        p2 = fmaT<T>(Arow[k + 2], v[(k + 2) * nr], p2);
        p3 = fmaT<T>(Arow[k + 3], v[(k + 3) * nr], p3);
    }
    return (p0 + p1) + (p2 + p3);
}

template <typename T, int M>
constexpr size_t bcr_factor_smem_bytes() {
    return sizeof(T) * (6 * Cta<T, M>::BLK + M) + sizeof(int) * M;
}

// One reduction step for kept row r = 2q by a cluster of two CTAs on two SMs
// (one CTA per SM holds the FP64 pipe about half busy on this work, so the
// two sides of the elimination are split): rank 0 inverts the left odd
// neighbour r-1 and forms alpha_q, alpha C_{r-1} and B' = alpha B_{r-1};
// rank 1 inverts the right odd neighbour r+1 (stored as Dinv[q]) and forms
// gamma_q, gamma B_{r+1} and C' = gamma C_{r+1}; after a cluster barrier rank 1
// reads alpha C_{r-1} from rank 0's shared memory and writes
// D' = D_r + alpha C_{r-1} + gamma B_{r+1}.  Each odd row is inverted by the
// clusters of both kept rows next to it (one launch and no grid-wide
// dependency per level).  With K == 1 rank 0 inverts the single row into Dinv[0].
template <typename T, typename TI, typename TO, int M>
__global__ void __cluster_dims__(2, 1, 1) __launch_bounds__(8 * M) k_bcr_factor(const BcrArgs a) {
    using S = Cta<T, M>;
    constexpr int BLK = S::BLK, LD = S::LD, R = S::R;
    constexpr long long MM = S::MM;
    namespace cg = cooperative_groups;
    cg::cluster_group cl = cg::this_cluster();
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T* sI = reinterpret_cast<T*>(smem_raw);   // block being inverted
    T* sO = sI + BLK;                         // B_r (rank 0) or C_r (rank 1)
    T* sP = sI + 2 * BLK;                     // C_{r-1} or B_{r+1}
    T* sQ = sI + 3 * BLK;                     // B_{r-1} or C_{r+1}
    T* sM = sI + 4 * BLK;                     // alpha or gamma
    T* sT = sI + 5 * BLK;                     // alpha C_{r-1} or gamma B_{r+1}
    T* colk = sI + 6 * BLK;
    int* perm = reinterpret_cast<int*>(colk + M);
    const TI* gB = static_cast<const TI*>(a.B);
    const TI* gD = static_cast<const TI*>(a.D);
    const TI* gC = static_cast<const TI*>(a.C);
    T* gDinv = static_cast<T*>(a.Dinv);
    const int g = (int)cl.block_rank();
    const Own<T, M> o;
    const long long q = blockIdx.x / 2;
    if (a.K == 1) {
        if (g == 0) {
            load_any<T, M>(sI, gD);
            __syncthreads();
            gj_inverse<T, M>(sI, colk, perm, a.status, a.level, -2, 0);
            store_blk<T, M>(gDinv, sI);
        }
        return;
    }
    const long long r = 2 * q;
    const bool has = (g == 0) ? (q >= 1) : (r + 1 < a.K);
    const bool hasQ = (g == 0) ? (r - 1 >= 1) : (r + 2 < a.K);
    T t[R], o2[R];
#pragma unroll
    for (int u = 0; u < R; ++u) t[u] = o2[u] = T(0);
    T* mult_out = static_cast<T*>(g == 0 ? a.al : a.ga) + q * MM;
    TO* o2_out = static_cast<TO*>(g == 0 ? a.Bn : a.Cn) + q * MM;
    if (has) {
        const long long nb = (g == 0) ? r - 1 : r + 1;
        load_any<T, M>(sI, gD + nb * MM);
        load_any<T, M>(sO, (g == 0 ? gB : gC) + r * MM);
        load_any<T, M>(sP, (g == 0 ? gC : gB) + nb * MM);
        if (hasQ) load_any<T, M>(sQ, (g == 0 ? gB : gC) + nb * MM);
        __syncthreads();
        gj_inverse<T, M>(sI, colk, perm, a.status, a.level, -2, nb);
        if (g == 1) store_blk<T, M>(gDinv + q * MM, sI);
        T mult[R];
#pragma unroll
        for (int u = 0; u < R; ++u) mult[u] = T(0);
        gemm_lat<T, M, true>(mult, sO, sI, o.r0, o.c);
        write_own<T, M>(sM, mult, o);
        store_own<T, M>(mult_out, mult, o);
        __syncthreads();
        gemm_lat<T, M, false>(t, sM, sP, o.r0, o.c);
        if (hasQ) gemm_lat<T, M, false>(o2, sM, sQ, o.r0, o.c);
    } else {
        T z[R];
        zero_own<T, M>(z);
        store_own<T, M>(mult_out, z, o);
    }
    store_own<T, M>(o2_out, o2, o);
    write_own<T, M>(sT, t, o);
    cl.sync();   // rank 0's alpha C_{r-1} is visible to rank 1
    if (g == 1) {
        const T* rT = cl.map_shared_rank(sT, 0);
        TO* gDn = static_cast<TO*>(a.Dn) + q * MM;
#pragma unroll
        for (int u = 0; u < R; ++u) {
            const int i = o.r0 + u;
            gDn[i * M + o.c] = (TO)((cvt_in<T>(gD[r * MM + i * M + o.c]) + rT[i * LD + o.c]) + t[u]);
        }
    }
    cl.sync();   // rank 0 keeps its shared memory until rank 1 has read it
}

template <typename T, int M>
constexpr size_t bcr_vec_smem_bytes() {
    return sizeof(T) * (3 * Cta<T, M>::BLK + 3 * M * 32);
}

// f'_q = f_{2q} + alpha_q f_{2q-1} + gamma_q f_{2q+1}; with K == 1: x = D^{-1} f.
template <typename T, int M>
__global__ void __launch_bounds__(8 * M) k_bcr_rhs(const BcrArgs a) {
    using S = Cta<T, M>;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T* s0 = reinterpret_cast<T*>(smem_raw);
    T* s1 = s0 + S::BLK;
    T* v0 = s1 + S::BLK;
    T* v1 = v0 + M * 32;
    const int nr = a.nr;
    const int E = M * nr;
    const long long q = blockIdx.x;
    const long long MM = S::MM;
    if (a.K == 1) {
        load_blkT<T, M>(s0, static_cast<const T*>(a.Dinv));
        for (int el = threadIdx.x; el < E; el += S::NT) v0[el] = cvt_in<T>(a.F[el]);
        __syncthreads();
        for (int el = threadIdx.x; el < E; el += S::NT) {
            const int rr = el / nr, c = el % nr;
            a.X[el] = (double)dot_lat<T, M>(s0 + rr * S::LD, v0 + c, nr);
        }
        return;
    }
    const long long r = 2 * q;
    const bool left = q >= 1, right = r + 1 < a.K;
    if (left) load_blkT<T, M>(s0, static_cast<const T*>(a.al) + q * MM);
    if (right) load_blkT<T, M>(s1, static_cast<const T*>(a.ga) + q * MM);
    for (int el = threadIdx.x; el < E; el += S::NT) {
        v0[el] = left ? cvt_in<T>(a.F[(r - 1) * E + el]) : T(0);
        v1[el] = right ? cvt_in<T>(a.F[(r + 1) * E + el]) : T(0);
    }
    __syncthreads();
    for (int el = threadIdx.x; el < E; el += S::NT) {
        const int rr = el / nr, c = el % nr;
        const T dl = left ? dot_lat<T, M>(s0 + rr * S::LD, v0 + c, nr) : T(0);
        const T dr = right ? dot_lat<T, M>(s1 + rr * S::LD, v1 + c, nr) : T(0);
        a.Fn[q * E + el] = a.F[r * E + el] + (double)(dl + dr);
    }
}

// x_{2q} = x'_q;  x_{2q+1} = D_{2q+1}^{-1} (f_{2q+1} - B_{2q+1} x'_q - C_{2q+1} x'_{q+1}).
template <typename T, typename TI, int M>
__global__ void __launch_bounds__(8 * M) k_bcr_back(const BcrArgs a) {
    using S = Cta<T, M>;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T* s0 = reinterpret_cast<T*>(smem_raw);
    T* s1 = s0 + S::BLK;
    T* s2 = s1 + S::BLK;
    T* v0 = s2 + S::BLK;
    T* v1 = v0 + M * 32;
    T* t = v1 + M * 32;
    const int nr = a.nr;
    const int E = M * nr;
    const long long q = blockIdx.x;
    const long long MM = S::MM;
    const long long r = 2 * q + 1;
    for (int el = threadIdx.x; el < E; el += S::NT) a.X[2 * q * E + el] = a.Xn[q * E + el];
    if (r >= a.K) return;
    const bool right = r + 1 < a.K;
    load_any<T, M>(s0, static_cast<const TI*>(a.B) + r * MM);
    if (right) load_any<T, M>(s1, static_cast<const TI*>(a.C) + r * MM);
    load_blkT<T, M>(s2, static_cast<const T*>(a.Dinv) + q * MM);
    for (int el = threadIdx.x; el < E; el += S::NT) {
        v0[el] = cvt_in<T>(a.Xn[q * E + el]);
        v1[el] = right ? cvt_in<T>(a.Xn[(q + 1) * E + el]) : T(0);
    }
    __syncthreads();
    for (int el = threadIdx.x; el < E; el += S::NT) {
        const int rr = el / nr, c = el % nr;
        const T bl = dot_lat<T, M>(s0 + rr * S::LD, v0 + c, nr);
        const T cr = right ? dot_lat<T, M>(s1 + rr * S::LD, v1 + c, nr) : T(0);
        t[el] = cvt_in<T>(a.F[r * E + el]) - (bl + cr);
    }
    __syncthreads();
    for (int el = threadIdx.x; el < E; el += S::NT) {
        const int rr = el / nr, c = el % nr;
        a.X[r * E + el] = (double)dot_lat<T, M>(s2 + rr * S::LD, t + c, nr);
    }
}

}  // namespace bt
