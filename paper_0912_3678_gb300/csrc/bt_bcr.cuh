// Block cyclic reduction (odd-even reduction) of the reduced system, the
// "cyclic reduction" variant of Sec. 2 applied to T_p with one
// synchronisation (kernel launch) per reduction step.  FP64, CTA per row
// (m >= 8).  Level l holds K active block rows (B_q, D_q, C_q, f_q); the rows
// at odd positions are eliminated:
//   alpha_q = -B_{2q} D_{2q-1}^{-1},  gamma_q = -C_{2q} D_{2q+1}^{-1}
//   D'_q = D_{2q} + alpha_q C_{2q-1} + gamma_q B_{2q+1}
//   B'_q = alpha_q B_{2q-1},  C'_q = gamma_q C_{2q+1},  f'_q = f_{2q} + alpha_q f_{2q-1} + gamma_q f_{2q+1}
// and after the single remaining row is solved the odd rows are recovered:
//   x_{2q+1} = D_{2q+1}^{-1} (f_{2q+1} - B_{2q+1} x_{2q} - C_{2q+1} x_{2q+2}).
#pragma once
#include <cooperative_groups.h>

#include "bt_cta.cuh"

namespace bt {

struct BcrArgs {
    long long K;          // active rows of this level
    int nr, level;
    const double* B;      // [K][m][m]
    const double* D;
    const double* C;
    double* Dinv;         // [K/2] inverses of the odd rows (the single row when K == 1)
    double* al;           // [(K+1)/2] alpha of the kept rows
    double* ga;           // [(K+1)/2] gamma of the kept rows
    double* Bn;           // next level [(K+1)/2][m][m]
    double* Dn;
    double* Cn;
    const double* F;      // [K][m][nr]
    double* Fn;           // [(K+1)/2][m][nr]
    double* X;            // [K][m][nr]
    const double* Xn;     // [(K+1)/2][m][nr]
    long long* status;
};

// The reduced levels are small, so these kernels are built for latency: each
// FP64 dot product of length M is split over four partial sums (dependency
// chains of M/4 instead of M), and one launch per level does the whole
// elimination step.

// acc[q] += sgn * (A B)[r0+q][c] over four partial sums.
template <int M, bool NEG>
__device__ __forceinline__ void gemm_lat(double (&acc)[M / 8], const double* A, const double* B, int r0, int c) {
    constexpr int LD = M + 1, R = M / 8;
    double p[R][4];
#pragma unroll
    for (int q = 0; q < R; ++q)
#pragma unroll
        for (int u = 0; u < 4; ++u) p[q][u] = 0.0;
#pragma unroll
    for (int k = 0; k < M; k += 4) {
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const double b = NEG ? -B[(k + u) * LD + c] : B[(k + u) * LD + c];
#pragma unroll
            for (int q = 0; q < R; ++q) p[q][u] = fma(A[(r0 + q) * LD + k + u], b, p[q][u]);
        }
    }
#pragma unroll
    for (int q = 0; q < R; ++q) acc[q] += (p[q][0] + p[q][1]) + (p[q][2] + p[q][3]);
}

// sum_k A[row][k] v[k * nr] over four partial sums (A in shared memory, row-padded).
template <int M>
__device__ __forceinline__ double dot_lat(const double* Arow, const double* v, int nr) {
    double p0 = 0.0, p1 = 0.0, p2 = 0.0, p3 = 0.0;
#pragma unroll
    for (int k = 0; k < M; k += 4) {
        p0 = fma(Arow[k], v[k * nr], p0);
        p1 = fma(Arow[k + 1], v[(k + 1) * nr], p1);
        p2 = fma(Arow[k + 2], v[(k + 2) * nr], p2);
        p3 = fma(Arow[k + 3], v[(k + 3) * nr], p3);
    }
    return (p0 + p1) + (p2 + p3);
}

template <int M>
constexpr size_t bcr_factor_smem_bytes() {
    return sizeof(double) * (6 * Cta<double, M>::BLK + M) + sizeof(int) * M;
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
template <int M>
__global__ void __cluster_dims__(2, 1, 1) __launch_bounds__(8 * M) k_bcr_factor(const BcrArgs a) {
    using S = Cta<double, M>;
    constexpr int NT = S::NT, BLK = S::BLK, LD = S::LD, R = S::R;
    constexpr long long MM = S::MM;
    namespace cg = cooperative_groups;
    cg::cluster_group cl = cg::this_cluster();
    extern __shared__ __align__(16) unsigned char smem_raw[];
    double* sI = reinterpret_cast<double*>(smem_raw);   // block being inverted
    double* sO = sI + BLK;                               // B_r (rank 0) or C_r (rank 1)
    double* sP = sI + 2 * BLK;                           // C_{r-1} or B_{r+1}
    double* sQ = sI + 3 * BLK;                           // B_{r-1} or C_{r+1}
    double* sM = sI + 4 * BLK;                           // alpha or gamma
    double* sT = sI + 5 * BLK;                           // alpha C_{r-1} or gamma B_{r+1}
    double* colk = sI + 6 * BLK;
    int* perm = reinterpret_cast<int*>(colk + M);
    const int g = (int)cl.block_rank();
    const Own<double, M> o;
    const long long q = blockIdx.x / 2;
    if (a.K == 1) {
        if (g == 0) {
            load_blk<double, M>(sI, a.D);
            __syncthreads();
            gj_inverse<double, M>(sI, colk, perm, a.status, a.level, -2, 0);
            store_blk<double, M>(a.Dinv, sI);
        }
        return;
    }
    const long long r = 2 * q;
    const bool has = (g == 0) ? (q >= 1) : (r + 1 < a.K);
    const bool hasQ = (g == 0) ? (r - 1 >= 1) : (r + 2 < a.K);
    double t[R], o2[R];
#pragma unroll
    for (int u = 0; u < R; ++u) t[u] = o2[u] = 0.0;
    double* mult_out = (g == 0 ? a.al : a.ga) + q * MM;
    double* o2_out = (g == 0 ? a.Bn : a.Cn) + q * MM;
    if (has) {
        const long long nb = (g == 0) ? r - 1 : r + 1;
        load_blk<double, M>(sI, a.D + nb * MM);
        load_blk<double, M>(sO, (g == 0 ? a.B : a.C) + r * MM);
        load_blk<double, M>(sP, (g == 0 ? a.C : a.B) + nb * MM);
        if (hasQ) load_blk<double, M>(sQ, (g == 0 ? a.B : a.C) + nb * MM);
        __syncthreads();
        gj_inverse<double, M>(sI, colk, perm, a.status, a.level, -2, nb);
        if (g == 1) store_blk<double, M>(a.Dinv + q * MM, sI);
        double mult[R];
#pragma unroll
        for (int u = 0; u < R; ++u) mult[u] = 0.0;
        gemm_lat<M, true>(mult, sO, sI, o.r0, o.c);
        write_own<double, M>(sM, mult, o);
        store_own<double, M>(mult_out, mult, o);
        __syncthreads();
        gemm_lat<M, false>(t, sM, sP, o.r0, o.c);
        if (hasQ) gemm_lat<M, false>(o2, sM, sQ, o.r0, o.c);
    } else {
        double z[R];
        zero_own<double, M>(z);
        store_own<double, M>(mult_out, z, o);
    }
    store_own<double, M>(o2_out, o2, o);
    write_own<double, M>(sT, t, o);
    cl.sync();   // rank 0's alpha C_{r-1} is visible to rank 1
    if (g == 1) {
        const double* rT = cl.map_shared_rank(sT, 0);
#pragma unroll
        for (int u = 0; u < R; ++u) {
            const int i = o.r0 + u;
            a.Dn[q * MM + i * M + o.c] = (a.D[r * MM + i * M + o.c] + rT[i * LD + o.c]) + t[u];
        }
    }
    cl.sync();   // rank 0 keeps its shared memory until rank 1 has read it
}

// f'_q = f_{2q} + alpha_q f_{2q-1} + gamma_q f_{2q+1}; with K == 1: x = D^{-1} f.
template <int M>
__global__ void __launch_bounds__(8 * M) k_bcr_rhs(const BcrArgs a) {
    using S = Cta<double, M>;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    double* s0 = reinterpret_cast<double*>(smem_raw);
    double* s1 = s0 + S::BLK;
    double* v0 = s1 + S::BLK;
    double* v1 = v0 + M * 32;
    const int nr = a.nr;
    const int E = M * nr;
    const long long q = blockIdx.x;
    const long long MM = S::MM;
    if (a.K == 1) {
        load_blk<double, M>(s0, a.Dinv);
        for (int el = threadIdx.x; el < E; el += S::NT) v0[el] = a.F[el];
        __syncthreads();
        for (int el = threadIdx.x; el < E; el += S::NT) {
            const int rr = el / nr, c = el % nr;
            a.X[el] = dot_lat<M>(s0 + rr * S::LD, v0 + c, nr);
        }
        return;
    }
    const long long r = 2 * q;
    const bool left = q >= 1, right = r + 1 < a.K;
    if (left) load_blk<double, M>(s0, a.al + q * MM);
    if (right) load_blk<double, M>(s1, a.ga + q * MM);
    for (int el = threadIdx.x; el < E; el += S::NT) {
        v0[el] = left ? a.F[(r - 1) * E + el] : 0.0;
        v1[el] = right ? a.F[(r + 1) * E + el] : 0.0;
    }
    __syncthreads();
    for (int el = threadIdx.x; el < E; el += S::NT) {
        const int rr = el / nr, c = el % nr;
        const double dl = left ? dot_lat<M>(s0 + rr * S::LD, v0 + c, nr) : 0.0;
        const double dr = right ? dot_lat<M>(s1 + rr * S::LD, v1 + c, nr) : 0.0;
        a.Fn[q * E + el] = a.F[r * E + el] + (dl + dr);
    }
}

// x_{2q} = x'_q;  x_{2q+1} = D_{2q+1}^{-1} (f_{2q+1} - B_{2q+1} x'_q - C_{2q+1} x'_{q+1}).
template <int M>
__global__ void __launch_bounds__(8 * M) k_bcr_back(const BcrArgs a) {
    using S = Cta<double, M>;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    double* s0 = reinterpret_cast<double*>(smem_raw);
    double* s1 = s0 + S::BLK;
    double* s2 = s1 + S::BLK;
    double* v0 = s2 + S::BLK;
    double* v1 = v0 + M * 32;
    double* t = v1 + M * 32;
    const int nr = a.nr;
    const int E = M * nr;
    const long long q = blockIdx.x;
    const long long MM = S::MM;
    const long long r = 2 * q + 1;
    for (int el = threadIdx.x; el < E; el += S::NT) a.X[2 * q * E + el] = a.Xn[q * E + el];
    if (r >= a.K) return;
    const bool right = r + 1 < a.K;
    load_blk<double, M>(s0, a.B + r * MM);
    if (right) load_blk<double, M>(s1, a.C + r * MM);
    load_blk<double, M>(s2, a.Dinv + q * MM);
    for (int el = threadIdx.x; el < E; el += S::NT) {
        v0[el] = a.Xn[q * E + el];
        v1[el] = right ? a.Xn[(q + 1) * E + el] : 0.0;
    }
    __syncthreads();
    for (int el = threadIdx.x; el < E; el += S::NT) {
        const int rr = el / nr, c = el % nr;
        const double bl = dot_lat<M>(s0 + rr * S::LD, v0 + c, nr);
        const double cr = right ? dot_lat<M>(s1 + rr * S::LD, v1 + c, nr) : 0.0;
        t[el] = a.F[r * E + el] - (bl + cr);
    }
    __syncthreads();
    for (int el = threadIdx.x; el < E; el += S::NT) {
        const int rr = el / nr, c = el % nr;
        a.X[r * E + el] = dot_lat<M>(s2 + rr * S::LD, t + c, nr);
    }
}

template <int M>
constexpr size_t bcr_vec_smem_bytes() {
    return sizeof(double) * (3 * Cta<double, M>::BLK + 3 * M * 32);
}

}  // namespace bt
