// Partition-method kernels with one CTA of 8*M threads per partition, for
// block sizes M in {8, 16, 32}.  All m x m block operations run from shared
// memory (rows padded to M+1 elements); thread t owns rows
// (t/M)*R .. (t/M)*R + R-1 of column t%M, R = M/8, so every GEMM keeps all
// lanes busy on the FP64 (or FP32) FMA pipe.
//
// Algorithm (Sec. 2, the LU-type parallel factorization, Eqs. (parfact)-(parblock),
// with the local block LU applied block row by block row and every pivot
// block D'_j inverted by Gauss-Jordan elimination with partial pivoting, the
// LUD/Gauss-Jordan form mentioned in Sec. 2):
//   forward over the local rows j of a partition:
//     D'_j  = D_j - B_j Y_{j-1}                (Schur complement update)
//     Y_j   = D'_j^{-1} C_j                    (fill-in of the upper factor)
//     Zc_j  = -D'_j^{-1} B_j Zc_{j-1}          (left spike; Zc_s = -D'_s^{-1} B_s)
//   so that x_j = h_j + Zc_j x_L - Y_j x_{j+1}; h_j = D'_j^{-1}(f_j - B_j h_{j-1}).
//   backward (full elimination, only the top row is kept):
//     P_j = Zc_j - Y_j P_{j+1},  Q_j = -Y_j Q_{j+1},  P_{e-1} = Zc_{e-1}, Q_{e-1} = -Y_{e-1}
//   giving x_first = H + P x_L + Q x_R.  The separator rows then form the
//   reduced matrix of Eq. (redmatr) (assembled by bt_assemble).
#pragma once
#include <cuda_bf16.h>
#include <type_traits>

#include "bt_device.cuh"
#include "bt_level.h"

namespace bt {

template <typename T, int M>
struct Cta {
    static constexpr int NT = 8 * M;
    static constexpr int LD = M + 1;
    static constexpr int R = M / 8;
    static constexpr int BLK = M * LD;
    static constexpr int MM = M * M;
};

// ------------------------------------------------------------ block moves --
template <typename T, int M>
__device__ __forceinline__ void load_blk(T* s, const double* g) {
    using S = Cta<T, M>;
    for (int idx = threadIdx.x; idx < M * M; idx += S::NT) s[(idx / M) * S::LD + idx % M] = (T)g[idx];
}
template <typename T, int M>
__device__ __forceinline__ void load_blkT(T* s, const T* g) {
    using S = Cta<T, M>;
    for (int idx = threadIdx.x; idx < M * M; idx += S::NT) s[(idx / M) * S::LD + idx % M] = g[idx];
}
template <typename T, int M, typename G>
__device__ __forceinline__ void store_blk(G* g, const T* s) {
    using S = Cta<T, M>;
    for (int idx = threadIdx.x; idx < M * M; idx += S::NT) g[idx] = (G)s[(idx / M) * S::LD + idx % M];
}

// Owned elements of thread t: rows r0+q (q < R), column c.
template <typename T, int M>
struct Own {
    int r0, c;
    __device__ __forceinline__ Own() : r0((threadIdx.x / M) * Cta<T, M>::R), c(threadIdx.x % M) {}
};

// acc[q] += sgn * (A B)[r0+q][c]
template <typename T, int M, bool NEG>
__device__ __forceinline__ void gemm_acc(T (&acc)[Cta<T, M>::R], const T* A, const T* B, const Own<T, M>& o) {
    using S = Cta<T, M>;
#pragma unroll 4
    for (int k = 0; k < M; ++k) {
        const T b = NEG ? -B[k * S::LD + o.c] : B[k * S::LD + o.c];
#pragma unroll
        for (int q = 0; q < S::R; ++q) acc[q] = fmaT<T>(A[(o.r0 + q) * S::LD + k], b, acc[q]);
    }
}

template <typename T, int M>
__device__ __forceinline__ void read_own(T (&v)[Cta<T, M>::R], const T* s, const Own<T, M>& o) {
#pragma unroll
    for (int q = 0; q < Cta<T, M>::R; ++q) v[q] = s[(o.r0 + q) * Cta<T, M>::LD + o.c];
}
template <typename T, int M>
__device__ __forceinline__ void write_own(T* s, const T (&v)[Cta<T, M>::R], const Own<T, M>& o) {
#pragma unroll
    for (int q = 0; q < Cta<T, M>::R; ++q) s[(o.r0 + q) * Cta<T, M>::LD + o.c] = v[q];
}
template <typename T, int M, typename G>
__device__ __forceinline__ void store_own(G* g, const T (&v)[Cta<T, M>::R], const Own<T, M>& o) {
#pragma unroll
    for (int q = 0; q < Cta<T, M>::R; ++q) g[(o.r0 + q) * M + o.c] = (G)v[q];
}
template <typename T, int M>
__device__ __forceinline__ void zero_own(T (&v)[Cta<T, M>::R]) {
#pragma unroll
    for (int q = 0; q < Cta<T, M>::R; ++q) v[q] = T(0);
}

// ------------------------------------------------------------ Gauss-Jordan --
// In-place inverse of the M x M block a (shared memory) by Gauss-Jordan
// elimination with partial pivoting.  Step k: one warp (warp k mod nwarps, so
// the serial work rotates over the SM sub-partitions) picks the pivot row p
// with the largest |a_ik|, i >= k (one redux over 32-bit keys: the top 26
// magnitude bits of each entry above the row index, so ties and magnitudes
// equal to 2^-20 relative go to the first row), swaps rows k and p, scales
// row k by 1/pivot and publishes the multiplier column; then every thread
// eliminates column k from its rows.  The row swaps are undone as column
// swaps at the end.  Reports a zero or non-finite pivot.  Entered and left
// with all threads synchronised.
template <typename T>
__device__ __forceinline__ unsigned mag_key(T v);
template <>
__device__ __forceinline__ unsigned mag_key<double>(double v) {
    return (unsigned)(__double2hiint(v) & 0x7fffffff) >> 5;
}
template <>
__device__ __forceinline__ unsigned mag_key<float>(float v) {
    return (__float_as_uint(v) & 0x7fffffffu) >> 5;
}
// A magnitude (truncated, never above it) back from its key.
template <typename T>
__device__ __forceinline__ T key_value(unsigned k);
template <>
__device__ __forceinline__ double key_value<double>(unsigned k) {
    return __hiloint2double((int)(k << 5), 0);
}
template <>
__device__ __forceinline__ float key_value<float>(unsigned k) {
    return __uint_as_float(k << 5);
}

// Pivoted levels pass brk: a pivot with |pivot| <= thr is then a breakdown of
// the partition's local factorization at this row (record_breakdown; the
// partition is split there), not an error.

template <typename T, int M>
__device__ bool gj_inverse(T* a, T* colk, int* perm, long long* st, int level, long long part,
                           long long row, long long* brk = nullptr, T thr = T(0), long long cap = 0) {
    using S = Cta<T, M>;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    constexpr int NW = S::NT / 32;
    const Own<T, M> o;
    bool ok = true;
    for (int k = 0; k < M; ++k) {
        if (warp == k % NW) {
            const T v = (lane < M) ? a[lane * S::LD + k] : T(0);
            const unsigned key = (lane >= k && lane < M) ? ((mag_key<T>(v) << 5) | (unsigned)(31 - lane)) : 0u;
            const unsigned best = __reduce_max_sync(0xffffffffu, key);
            const int p = 31 - (int)(best & 31u);
            T pv = __shfl_sync(0xffffffffu, v, p);
            const T vk = __shfl_sync(0xffffffffu, v, k);
            if (nonfinite(pv)) {
                if (lane == 0) report(st, ST_NONFINITE, level, part, row);
                pv = T(1);
                ok = false;
            } else if (brk != nullptr && !(abs_key(pv) > abs_key(thr))) {
                if (lane == 0) record_breakdown(brk, cap, row);
                pv = T(1);
                ok = false;
            } else if (pv == T(0)) {
                if (lane == 0) report(st, ST_SINGULAR, level, part, row);
                pv = T(1);
                ok = false;
            }
            const T r = rcp(pv);
            if (lane < M) {
                colk[lane] = (lane == k) ? T(0) : (lane == p ? vk : v);
                const T tk = a[k * S::LD + lane];
                const T tp = a[p * S::LD + lane];
                a[p * S::LD + lane] = tk;
                a[k * S::LD + lane] = (lane == k) ? r : tp * r;
            }
            if (lane == 0) perm[k] = p;
        }
        __syncthreads();
#pragma unroll
        for (int q = 0; q < S::R; ++q) {
            const int i = o.r0 + q;
            if (i != k) {
                const T l = colk[i];
                const T akc = a[k * S::LD + o.c];
                a[i * S::LD + o.c] = (o.c == k) ? -l * akc : fmaT<T>(-l, akc, a[i * S::LD + o.c]);
            }
        }
        __syncthreads();
    }
    if (warp == 0 && lane < M) {
        for (int k = M - 1; k >= 0; --k) {
            const int p = perm[k];
            if (p != k) {
                const T t = a[lane * S::LD + k];
                a[lane * S::LD + k] = a[lane * S::LD + p];
                a[lane * S::LD + p] = t;
            }
        }
    }
    __syncthreads();
    return ok;
}

// ------------------------------------------------------ BF16 tensor cores --
// P = A B for M x M FP32 blocks in shared memory, with the operands rounded
// to BF16 and FP32 accumulation, by warp-level mma.sync m16n8k16 tiles
// (row-major A, column-major B fragments).  Tiles are spread over the warps.
__device__ __forceinline__ unsigned pack_bf16(float lo, float hi) {
    const __nv_bfloat162 v = __floats2bfloat162_rn(lo, hi);
    return *reinterpret_cast<const unsigned*>(&v);
}

template <int M>
__device__ __forceinline__ void gemm_bf16_tc(float* P, const float* A, const float* B) {
    constexpr int LD = M + 1;
    constexpr int MT = M / 16, NTL = M / 8, KS = M / 16;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
    const int g = lane >> 2, t = lane & 3;
    for (int tile = warp; tile < MT * NTL; tile += nwarps) {
        const int mt = tile / NTL, nt = tile % NTL;
        float c0 = 0.f, c1 = 0.f, c2 = 0.f, c3 = 0.f;
#pragma unroll
        for (int ks = 0; ks < KS; ++ks) {
            const int r0 = mt * 16 + g, k0 = ks * 16 + 2 * t, n0 = nt * 8 + g;
            const unsigned a0 = pack_bf16(A[r0 * LD + k0], A[r0 * LD + k0 + 1]);
            const unsigned a1 = pack_bf16(A[(r0 + 8) * LD + k0], A[(r0 + 8) * LD + k0 + 1]);
            const unsigned a2 = pack_bf16(A[r0 * LD + k0 + 8], A[r0 * LD + k0 + 9]);
            const unsigned a3 = pack_bf16(A[(r0 + 8) * LD + k0 + 8], A[(r0 + 8) * LD + k0 + 9]);
            const unsigned b0 = pack_bf16(B[k0 * LD + n0], B[(k0 + 1) * LD + n0]);
            const unsigned b1 = pack_bf16(B[(k0 + 8) * LD + n0], B[(k0 + 9) * LD + n0]);
            asm volatile(
                "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
                "{%0,%1,%2,%3};"
                : "+f"(c0), "+f"(c1), "+f"(c2), "+f"(c3)
                : "r"(a0), "r"(a1), "r"(a2), "r"(a3), "r"(b0), "r"(b1));
        }
        const int r = mt * 16 + g, c = nt * 8 + 2 * t;
        P[r * LD + c] = c0;
        P[r * LD + c + 1] = c1;
        P[(r + 8) * LD + c] = c2;
        P[(r + 8) * LD + c + 1] = c3;
    }
}

template <typename T, int M>
constexpr size_t factor_smem_bytes() {
    return sizeof(T) * (7 * Cta<T, M>::BLK + M) + sizeof(int) * M;
}

// ------------------------------------------------------------------ factor --
// One CTA per partition.  Mode 0: block tridiagonal level; mode 1: BABD level
// (C = 0, so Y = 0 and no backward sweep; the right separator's reduced row
// of Eq. (redmatr1) is written here: S'[i] = B_e Zc_{e-1}, R'[i] = D_e).
// Per-thread prefetch of the next block row (R elements of each of B, D, C),
// issued before the current row's work and stored to shared memory after it.
template <typename T, int M>
struct RowPrefetch {
    double b[Cta<T, M>::R], d[Cta<T, M>::R], c[Cta<T, M>::R];
    __device__ __forceinline__ void load(const double* gB, const double* gD, const double* gC) {
#pragma unroll
        for (int u = 0; u < Cta<T, M>::R; ++u) {
            const int idx = threadIdx.x + u * Cta<T, M>::NT;
            d[u] = gD[idx];
            if (gB) b[u] = gB[idx];
            if (gC) c[u] = gC[idx];
        }
    }
    __device__ __forceinline__ void store(T* sB, T* sD, T* sC, bool hasB, bool hasC) const {
        using S = Cta<T, M>;
#pragma unroll
        for (int u = 0; u < S::R; ++u) {
            const int idx = threadIdx.x + u * S::NT;
            const int at = (idx / M) * S::LD + idx % M;
            sD[at] = (T)d[u];
            if (hasB) sB[at] = (T)b[u];
            if (hasC) sC[at] = (T)c[u];
        }
    }
};

// One CTA per partition.  Mode 0: block tridiagonal level; the top-row
// coupling that the reduced row of the left separator needs is accumulated
// during the forward sweep: with W_s = C_sep (the left separator row's block
// coupling it to x_s) and W_{j+1} = -W_j Y_j,
//   C_sep P_first = sum_j W_j Zc_j   (stored in Pf)  and  C_sep Q_first = W_e (Qf),
// where x_first = H + P_first x_L + Q_first x_R after full elimination.
// Mode 1: BABD level (C = 0, so Y = 0); the right separator's reduced row of
// Eq. (redmatr1) is written here: S'[i] = B_e Zc_{e-1}, R'[i] = D_e.
template <typename T, int M, int MODE>
__device__ __forceinline__ void factor_cta_body(const LevelArgs& a, const long long i, unsigned char* smem_raw) {
    using S = Cta<T, M>;
    T* sB = reinterpret_cast<T*>(smem_raw);
    T* sD = sB + S::BLK;
    T* sC = sD + S::BLK;
    T* sY = sC + S::BLK;
    T* sZ = sY + S::BLK;
    T* sT = sZ + S::BLK;
    T* sW = sT + S::BLK;
    T* colk = sW + S::BLK;
    int* perm = reinterpret_cast<int*>(colk + M);

    const Part pt = part_bounds(a, MODE, i);
    const Own<T, M> o;
    T* gDinv = reinterpret_cast<T*>(a.Dinv);
    T* gY = reinterpret_cast<T*>(a.Y);
    T* gZ = reinterpret_cast<T*>(a.Zc);
    const long long MM = S::MM;
    const bool wchain = (MODE == 0) && pt.hasL;
    T cp[S::R];   // sum_j W_j Zc_j (own elements)
    zero_own<T, M>(cp);

    auto needB = [&](long long j) { return j > pt.s || pt.hasL; };
    auto needC = [&](long long j) { return (MODE == 0) && ((j < pt.e - 1) || pt.hasR); };
    // rows of this launch: the whole partition, or one phase of it (the rows of every
    // partition arriving in slabs); a later phase resumes from the state the previous
    // one left in Y, Zc (rows already stored) and Pf, Qf (the running sum and W)
    long long jb = pt.s, je = pt.e;
    const bool phased = (MODE == 0) && a.phases > 1;
    if (phased) {
        const long long cnt = pt.e - pt.s;
        jb = pt.s + cnt * a.phase / a.phases;
        je = pt.s + cnt * (a.phase + 1) / a.phases;
    }
    if (jb < je) {
        RowPrefetch<T, M> pf;
        pf.load(needB(jb) ? a.B + (jb - a.shift) * MM : nullptr, a.D + (jb - a.shift) * MM,
                needC(jb) ? a.C + (jb - a.shift) * MM : nullptr);
        pf.store(sB, sD, sC, needB(jb), needC(jb));
    }
    if (jb > pt.s) {
        if (jb < je) {
            load_blkT<T, M>(sY, gY + (jb - 1) * MM);
            if (pt.hasL) load_blkT<T, M>(sZ, gZ + (jb - 1) * MM);
        }
        if (wchain) {
            load_blkT<T, M>(sW, reinterpret_cast<const T*>(a.Qf) + i * MM);
            const T* gP = reinterpret_cast<const T*>(a.Pf) + i * MM;
#pragma unroll
            for (int q = 0; q < S::R; ++q) cp[q] = gP[(o.r0 + q) * M + o.c];
        }
    } else if (wchain) {
        load_blk<T, M>(sW, a.C + (pt.s - 1 - a.shift) * MM);   // W_s = C of the left separator row
    }
    __syncthreads();

    for (long long j = jb; j < je; ++j) {
        const bool first = (j == pt.s);
        const bool nC = needC(j);
        const bool more = (j + 1 < je);
        RowPrefetch<T, M> pf;
        if (more)
            pf.load(needB(j + 1) ? a.B + (j + 1 - a.shift) * MM : nullptr, a.D + (j + 1 - a.shift) * MM,
                    needC(j + 1) ? a.C + (j + 1 - a.shift) * MM : nullptr);
        if (!first) {
            T acc[S::R];
            if (MODE == 0) {
                bool done = false;
                if constexpr (std::is_same<T, float>::value && M >= 16) {
                    if (a.bf16) {
                        gemm_bf16_tc<M>(sT, sB, sY);
                        __syncthreads();
                        T pr[S::R];
                        read_own<T, M>(acc, sD, o);
                        read_own<T, M>(pr, sT, o);
#pragma unroll
                        for (int u = 0; u < S::R; ++u) acc[u] -= pr[u];
                        done = true;
                    }
                }
                if (!done) {
                    read_own<T, M>(acc, sD, o);
                    gemm_acc<T, M, true>(acc, sB, sY, o);
                }
            }
            // the left-spike product t = B_j Zc_{j-1} does not need D'_j: take it here
            if (pt.hasL) {
                T t[S::R];
                zero_own<T, M>(t);
                gemm_acc<T, M, false>(t, sB, sZ, o);
                __syncthreads();
                write_own<T, M>(sT, t, o);
            }
            if (MODE == 0) write_own<T, M>(sD, acc, o);
            __syncthreads();
        }
        T thr = T(0);
        if (a.brk != nullptr) {
            // breakdown threshold: tau times the largest entry of B_j, D'_j, C_j
            unsigned mk = 0u;
#pragma unroll
            for (int q = 0; q < S::R; ++q) {
                const int at = (o.r0 + q) * S::LD + o.c;
                mk = max(mk, mag_key<T>(sD[at]));
                if (needB(j)) mk = max(mk, mag_key<T>(sB[at]));
                if (nC) mk = max(mk, mag_key<T>(sC[at]));
            }
            mk = __reduce_max_sync(0xffffffffu, mk);
            unsigned* red = reinterpret_cast<unsigned*>(perm);
            if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = mk;
            __syncthreads();
            unsigned bm = 0u;
            for (int w = 0; w < S::NT / 32; ++w) bm = max(bm, red[w]);
            __syncthreads();
            thr = (T)a.tau * key_value<T>(bm);
        }
        const bool ok = gj_inverse<T, M>(sD, colk, perm, a.status, a.level, i, j, a.brk, thr, a.brk_cap);
        // after a breakdown the local factorization restarts at the next row (as
        // if this row were a separator), so one pass finds every breakdown
        const bool restart = (a.brk != nullptr) && __syncthreads_or(!ok);
        store_blk<T, M>(gDinv + j * MM, sD);
        T z[S::R], y[S::R];
        if (pt.hasL) {
            zero_own<T, M>(z);
            gemm_acc<T, M, true>(z, sD, first ? sB : sT, o);
        }
        if (nC) {
            zero_own<T, M>(y);
            gemm_acc<T, M, false>(y, sD, sC, o);
        }
        __syncthreads();
        if (pt.hasL) {
            write_own<T, M>(sZ, z, o);
            store_own<T, M>(gZ + j * MM, z, o);
        }
        if (nC) {
            if (restart) zero_own<T, M>(y);
            write_own<T, M>(sY, y, o);
            store_own<T, M>(gY + j * MM, y, o);
        }
        __syncthreads();
        if (wchain) {
            // cp += W_j Zc_j ;  W_{j+1} = -W_j Y_j
            gemm_acc<T, M, false>(cp, sW, sZ, o);
            T wn[S::R];
            zero_own<T, M>(wn);
            if (nC) gemm_acc<T, M, true>(wn, sW, sY, o);
            __syncthreads();
            write_own<T, M>(sW, wn, o);
        }
        if (more) pf.store(sB, sD, sC, needB(j + 1), needC(j + 1));
        __syncthreads();
    }

    if (MODE == 0) {
        if (!pt.hasL) return;
        // final: C_sep P_first and W_e; between phases: the running sum and W
        store_own<T, M>(reinterpret_cast<T*>(a.Pf) + i * MM, cp, o);
        store_blk<T, M>(reinterpret_cast<T*>(a.Qf) + i * MM, sW);   // W_e (zero when there is no x_R)
    } else {
        // BABD: reduced row i+1 couples separator e to the left separator
        const long long e = pt.e;
        load_blk<T, M>(sB, a.B + (e - a.shift) * MM);
        __syncthreads();
        double* Sn = a.Bn + i * MM;
        double* Rn = a.Dn + i * MM;
        for (int idx = threadIdx.x; idx < M * M; idx += S::NT) Rn[idx] = a.D[(e - a.shift) * MM + idx];
        if (pt.e > pt.s) {
            T acc[S::R];
            zero_own<T, M>(acc);
            gemm_acc<T, M, false>(acc, sB, sZ, o);
            store_own<T, M>(Sn, acc, o);
        } else {
            for (int idx = threadIdx.x; idx < M * M; idx += S::NT) Sn[idx] = a.B[(e - a.shift) * MM + idx];
        }
    }
}

// ---------------------------------------------------------------- assemble --
// Block tridiagonal: the reduced row of separator s (the last row e of
// partition s) in FP64:
//   alpha = D_e - B_e Y_{e-1} + C_e P^(s+1)_first,  beta = B_e Zc_{e-1} (s > 0),
//   gamma = C_e Q^(s+1)_first (s+1 < p-1),
// where the factor kernel left C_e P_first and C_e Q_first of partition s+1 in
// Pf and Qf.
template <typename T, int M>
__device__ __forceinline__ void assemble_cta_body(const LevelArgs& a, const long long s, unsigned char* smem_raw) {
    using S = Cta<double, M>;
    double* sB = reinterpret_cast<double*>(smem_raw);
    double* sY = sB + S::BLK;
    double* sZ = sY + S::BLK;
    const Part pt = part_bounds(a, 0, s);
    const long long e = pt.e;
    const long long MM = S::MM;
    const Own<double, M> o;
    const bool hasBeta = s > 0;
    const bool hasGamma = (s + 1) < a.p - 1;
    const bool local = pt.e > pt.s;   // partition s has local rows before its separator
    load_blk<double, M>(sB, a.B + (e - a.shift) * MM);
    if (local) {
        const T* gY = reinterpret_cast<const T*>(a.Y) + (e - 1) * MM;
        for (int idx = threadIdx.x; idx < M * M; idx += S::NT) sY[(idx / M) * S::LD + idx % M] = (double)gY[idx];
        if (hasBeta) {
            const T* gZ = reinterpret_cast<const T*>(a.Zc) + (e - 1) * MM;
            for (int idx = threadIdx.x; idx < M * M; idx += S::NT) sZ[(idx / M) * S::LD + idx % M] = (double)gZ[idx];
        }
    }
    __syncthreads();
    const T* gP = reinterpret_cast<const T*>(a.Pf) + (s + 1) * MM;
    const T* gQ = reinterpret_cast<const T*>(a.Qf) + (s + 1) * MM;
    double al[S::R], be[S::R], ga[S::R];
#pragma unroll
    for (int q = 0; q < S::R; ++q) {
        const long long at = (o.r0 + q) * M + o.c;
        al[q] = a.D[(e - a.shift) * MM + at] + (double)gP[at];
        ga[q] = hasGamma ? (double)gQ[at] : 0.0;
        be[q] = 0.0;
    }
    if (local) {
        gemm_acc<double, M, true>(al, sB, sY, o);
        if (hasBeta) gemm_acc<double, M, false>(be, sB, sZ, o);
    } else if (hasBeta) {
        read_own<double, M>(be, sB, o);   // the separator couples directly to the previous one
    }
    store_own<double, M>(a.Dn + s * MM, al, o);
    store_own<double, M>(a.Bn + s * MM, be, o);
    store_own<double, M>(a.Cn + s * MM, ga, o);
}

// ------------------------------------------------------------------- solve --
// Elements of an M x nr right-hand-side block owned by thread t: t + u*NT.
template <int M>
struct RhsOwn {
    static constexpr int MAXU = 4;   // nr <= 32
};

// Forward substitution h_j = D'_j^{-1}(f_j - B_j h_{j-1}); h_j is written to X.
// Mode 0 with a left separator: backward H_j = h_j - Y_j H_{j+1} to the top row
// (Hf).  Mode 1: the right separator's reduced right-hand side
// g = f_e - B_e h_{e-1} (and partition 0 copies the boundary row).
template <typename T, int M, int MODE>
__device__ __forceinline__ void solve_fwd_cta_body(const LevelArgs& a, const long long i, unsigned char* smem_raw) {
    using S = Cta<T, M>;
    constexpr int NT = S::NT;
    T* sB = reinterpret_cast<T*>(smem_raw);
    T* sD = sB + S::BLK;
    T* sh = sD + S::BLK;          // M x nr
    T* sv = sh + M * 32;          // M x nr
    const int nr = a.nr;
    const int E = M * nr;
    const Part pt = part_bounds(a, MODE, i);
    const long long MM = S::MM;
    const T* gDinv = reinterpret_cast<const T*>(a.Dinv);
    constexpr int RU = RhsOwn<M>::MAXU;
    // per-thread prefetch of the next row: D'^{-1} (R), B (R), f (RU)
    T pD[S::R];
    double pB[S::R], pf[RU];
    auto fetch = [&](long long j) {
#pragma unroll
        for (int u = 0; u < S::R; ++u) {
            const int idx = threadIdx.x + u * NT;
            pD[u] = gDinv[j * MM + idx];
            pB[u] = (j > pt.s) ? a.B[(j - a.shift) * MM + idx] : 0.0;
        }
#pragma unroll
        for (int u = 0; u < RU; ++u) {
            const int el = threadIdx.x + u * NT;
            pf[u] = (el < E) ? a.F[j * E + el] : 0.0;
        }
    };
    auto stash = [&]() {
#pragma unroll
        for (int u = 0; u < S::R; ++u) {
            const int idx = threadIdx.x + u * NT;
            const int at = (idx / M) * S::LD + idx % M;
            sD[at] = pD[u];
            sB[at] = (T)pB[u];
        }
#pragma unroll
        for (int u = 0; u < RU; ++u) {
            const int el = threadIdx.x + u * NT;
            if (el < E) sv[el] = (T)pf[u];
        }
    };
    if (pt.s < pt.e) {
        fetch(pt.s);
        stash();
    }
    __syncthreads();
    for (long long j = pt.s; j < pt.e; ++j) {
        const bool first = (j == pt.s);
        const bool more = (j + 1 < pt.e);
        if (more) fetch(j + 1);
        if (!first) {
            for (int el = threadIdx.x; el < E; el += NT) {
                const int r = el / nr, c = el % nr;
                T acc = sv[el];
#pragma unroll 8
                for (int k = 0; k < M; ++k) acc = fmaT<T>(-sB[r * S::LD + k], sh[k * nr + c], acc);
                sv[el] = acc;
            }
            __syncthreads();
        }
        T h[RU];
#pragma unroll
        for (int u = 0; u < RU; ++u) {
            const int el = threadIdx.x + u * NT;
            h[u] = T(0);
            if (el < E) {
                const int r = el / nr, c = el % nr;
                T acc = T(0);
#pragma unroll 8
                for (int k = 0; k < M; ++k) acc = fmaT<T>(sD[r * S::LD + k], sv[k * nr + c], acc);
                h[u] = acc;
            }
        }
        __syncthreads();
#pragma unroll
        for (int u = 0; u < RU; ++u) {
            const int el = threadIdx.x + u * NT;
            if (el < E) {
                sh[el] = h[u];
                a.X[j * E + el] = (double)h[u];
            }
        }
        if (more) stash();
        __syncthreads();
    }
    if (MODE == 1) {
        const long long e = pt.e;
        if (i == 0)
            for (int el = threadIdx.x; el < E; el += NT) a.Fn[el] = a.F[el];
        load_blk<T, M>(sB, a.B + (e - a.shift) * MM);
        __syncthreads();
        for (int el = threadIdx.x; el < E; el += NT) {
            const int r = el / nr, c = el % nr;
            double acc = a.F[e * E + el];
            if (pt.e > pt.s) {
                T t = T(0);
#pragma unroll 8
                for (int k = 0; k < M; ++k) t = fmaT<T>(sB[r * S::LD + k], sh[k * nr + c], t);
                acc -= (double)t;
            }
            a.Fn[(i + 1) * E + el] = acc;
        }
        return;
    }
    if (!pt.hasL) return;
    if (pt.e == pt.s) {
        // no local rows: nothing between the two separators
        T* Hf = reinterpret_cast<T*>(a.Hf) + i * E;
        for (int el = threadIdx.x; el < E; el += NT) Hf[el] = T(0);
        return;
    }
    const T* gY = reinterpret_cast<const T*>(a.Y);
    for (long long j = pt.e - 2; j >= pt.s; --j) {
        load_blkT<T, M>(sB, gY + j * MM);
        for (int el = threadIdx.x; el < E; el += NT) sv[el] = (T)a.X[j * E + el];
        __syncthreads();
        T h[RhsOwn<M>::MAXU];
#pragma unroll
        for (int u = 0; u < RhsOwn<M>::MAXU; ++u) {
            const int el = threadIdx.x + u * NT;
            h[u] = T(0);
            if (el < E) {
                const int r = el / nr, c = el % nr;
                T acc = sv[el];
#pragma unroll 8
                for (int k = 0; k < M; ++k) acc = fmaT<T>(-sB[r * S::LD + k], sh[k * nr + c], acc);
                h[u] = acc;
            }
        }
        __syncthreads();
#pragma unroll
        for (int u = 0; u < RhsOwn<M>::MAXU; ++u) {
            const int el = threadIdx.x + u * NT;
            if (el < E) sh[el] = h[u];
        }
        __syncthreads();
    }
    T* Hf = reinterpret_cast<T*>(a.Hf) + i * E;
    for (int el = threadIdx.x; el < E; el += NT) Hf[el] = sh[el];
}

// Block tridiagonal reduced right-hand side of separator s:
//   g = f_e - B_e h_{e-1} - C_e H^(s+1)_first   (FP64).
template <typename T, int M>
__device__ __forceinline__ void assemble_rhs_cta_body(const LevelArgs& a, const long long s,
                                                      unsigned char* smem_raw) {
    using S = Cta<double, M>;
    constexpr int NT = S::NT;
    double* sB = reinterpret_cast<double*>(smem_raw);
    double* sC = sB + S::BLK;
    double* sh = sC + S::BLK;
    double* sH = sh + M * 32;
    const int nr = a.nr;
    const int E = M * nr;
    const Part pt = part_bounds(a, 0, s);
    const long long e = pt.e;
    const long long MM = S::MM;
    load_blk<double, M>(sB, a.B + (e - a.shift) * MM);
    load_blk<double, M>(sC, a.C + (e - a.shift) * MM);
    const T* Hf = reinterpret_cast<const T*>(a.Hf) + (s + 1) * E;
    const bool local = pt.e > pt.s;
    for (int el = threadIdx.x; el < E; el += NT) {
        sh[el] = local ? a.X[(e - 1) * E + el] : 0.0;
        sH[el] = (double)Hf[el];
    }
    __syncthreads();
    for (int el = threadIdx.x; el < E; el += NT) {
        const int r = el / nr, c = el % nr;
        double acc = a.F[e * E + el];
#pragma unroll 8
        for (int k = 0; k < M; ++k) {
            acc = fma(-sB[r * S::LD + k], sh[k * nr + c], acc);
            acc = fma(-sC[r * S::LD + k], sH[k * nr + c], acc);
        }
        a.Fn[s * E + el] = acc;
    }
}

// Back substitution x_j = h_j + Zc_j x_L - Y_j x_{j+1} from the last local row
// up, with x_L, x_R from the next level's solution; also copies the
// separator rows owned by this partition into X.
template <typename T, int M, int MODE>
__device__ __forceinline__ void solve_bwd_cta_body(const LevelArgs& a, const long long i, unsigned char* smem_raw) {
    using S = Cta<T, M>;
    constexpr int NT = S::NT;
    T* sY = reinterpret_cast<T*>(smem_raw);
    T* sZ = sY + S::BLK;
    T* sx = sZ + S::BLK;   // x_{j+1}
    T* sL = sx + M * 32;   // x_L
    const int nr = a.nr;
    const int E = M * nr;
    const Part pt = part_bounds(a, MODE, i);
    const long long MM = S::MM;
    const long long li = (MODE == 0) ? i - 1 : i;   // next-level index of x_L
    const long long ri = (MODE == 0) ? i : i + 1;   // next-level index of x_R
    for (int el = threadIdx.x; el < E; el += NT) {
        const double xr = pt.hasR ? a.Xn[ri * E + el] : 0.0;
        sx[el] = (T)xr;
        sL[el] = pt.hasL ? (T)a.Xn[li * E + el] : T(0);
        if (pt.hasR) a.X[pt.e * E + el] = xr;
        if (MODE == 1 && i == 0) a.X[el] = a.Xn[el];
    }
    __syncthreads();
    const T* gY = reinterpret_cast<const T*>(a.Y);
    const T* gZ = reinterpret_cast<const T*>(a.Zc);
    constexpr int RU = RhsOwn<M>::MAXU;
    T pY[S::R], pZ[S::R];
    double ph[RU];
    auto useY = [&](long long j) { return (MODE == 0) && ((j < pt.e - 1) || pt.hasR); };
    auto fetch = [&](long long j) {
#pragma unroll
        for (int u = 0; u < S::R; ++u) {
            const int idx = threadIdx.x + u * NT;
            pY[u] = useY(j) ? gY[j * MM + idx] : T(0);
            pZ[u] = pt.hasL ? gZ[j * MM + idx] : T(0);
        }
#pragma unroll
        for (int u = 0; u < RU; ++u) {
            const int el = threadIdx.x + u * NT;
            ph[u] = (el < E) ? a.X[j * E + el] : 0.0;
        }
    };
    auto stash = [&]() {
#pragma unroll
        for (int u = 0; u < S::R; ++u) {
            const int idx = threadIdx.x + u * NT;
            const int at = (idx / M) * S::LD + idx % M;
            sY[at] = pY[u];
            sZ[at] = pZ[u];
        }
    };
    if (pt.e > pt.s) {
        fetch(pt.e - 1);
        stash();
    }
    __syncthreads();
    for (long long j = pt.e - 1; j >= pt.s; --j) {
        const bool uY = useY(j);
        const bool more = (j - 1 >= pt.s);
        double hcur[RU];
#pragma unroll
        for (int u = 0; u < RU; ++u) hcur[u] = ph[u];
        if (more) fetch(j - 1);
        T xv[RU];
#pragma unroll
        for (int u = 0; u < RU; ++u) {
            const int el = threadIdx.x + u * NT;
            xv[u] = T(0);
            if (el < E) {
                const int r = el / nr, c = el % nr;
                T acc = (T)hcur[u];
                if (uY) {
#pragma unroll 8
                    for (int k = 0; k < M; ++k) acc = fmaT<T>(-sY[r * S::LD + k], sx[k * nr + c], acc);
                }
                if (pt.hasL) {
#pragma unroll 8
                    for (int k = 0; k < M; ++k) acc = fmaT<T>(sZ[r * S::LD + k], sL[k * nr + c], acc);
                }
                xv[u] = acc;
            }
        }
        __syncthreads();
#pragma unroll
        for (int u = 0; u < RU; ++u) {
            const int el = threadIdx.x + u * NT;
            if (el < E) {
                sx[el] = xv[u];
                a.X[j * E + el] = (double)xv[u];
            }
        }
        if (more) stash();
        __syncthreads();
    }
}

// ---------------------------------------------------------------- wrappers --
// Single system: CTA b handles partition b.  Batched (persistent): CTA b
// handles work items b, b + gridDim.x, ... where item w is (system, partition)
// = work[w] and the system's level is args[work[w].x].
#define BT_CTA_KERNELS(NAME, BODY, TPL, TARGS)                                                          \
    template <TPL>                                                                                     \
    __global__ void __launch_bounds__(8 * M) NAME(const LevelArgs a) {                                 \
        extern __shared__ __align__(16) unsigned char smem_raw[];                                      \
        const long long u = a.unit0 + (long long)blockIdx.x;                                           \
        if (a.unit_end > 0 && u >= a.unit_end) return;                                                 \
        BODY<TARGS>(a, u, smem_raw);                                                                   \
    }                                                                                                  \
    template <TPL>                                                                                     \
    __global__ void __launch_bounds__(8 * M)                                                           \
        NAME##_batch(const LevelArgs* __restrict__ args, const int2* __restrict__ work, int nwork) {   \
        extern __shared__ __align__(16) unsigned char smem_raw[];                                      \
        for (int w = blockIdx.x; w < nwork; w += gridDim.x) {                                           \
            const int2 it = work[w];                                                                   \
            const LevelArgs a = args[it.x];                                                            \
            BODY<TARGS>(a, (long long)it.y, smem_raw);                                                  \
            __syncthreads();                                                                           \
        }                                                                                              \
    }

#define BT_COMMA ,
BT_CTA_KERNELS(k_factor_cta, factor_cta_body, typename T BT_COMMA int M BT_COMMA int MODE, T BT_COMMA M BT_COMMA MODE)
BT_CTA_KERNELS(k_assemble_cta, assemble_cta_body, typename T BT_COMMA int M, T BT_COMMA M)
BT_CTA_KERNELS(k_solve_fwd_cta, solve_fwd_cta_body, typename T BT_COMMA int M BT_COMMA int MODE, T BT_COMMA M BT_COMMA MODE)
BT_CTA_KERNELS(k_assemble_rhs_cta, assemble_rhs_cta_body, typename T BT_COMMA int M, T BT_COMMA M)
BT_CTA_KERNELS(k_solve_bwd_cta, solve_bwd_cta_body, typename T BT_COMMA int M BT_COMMA int MODE, T BT_COMMA M BT_COMMA MODE)

template <typename T, int M>
constexpr size_t solve_smem_bytes() {
    return sizeof(T) * (2 * Cta<T, M>::BLK + 2 * M * 32);
}
template <int M>
constexpr size_t assemble_smem_bytes() {
    return sizeof(double) * (3 * Cta<double, M>::BLK);
}
template <int M>
constexpr size_t assemble_rhs_smem_bytes() {
    return sizeof(double) * (2 * Cta<double, M>::BLK + 2 * M * 32);
}

}  // namespace bt
