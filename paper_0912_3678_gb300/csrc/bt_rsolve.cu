// Solve of the reduced system (Eq. (redmatr)) by block cyclic reduction in one
// launch, for the refined paths: the cyclic-reduction factors (computed by
// k_bcr_factor, Sec. 2 cyclic-reduction variant) are applied in FP32 inside
// the FP32 correction solve that the FP64 refinement corrects.  One
// thread-block cluster (16 CTAs where the device can place such a cluster,
// else 8) runs every level:
//   forward   f^{q+1}_i = f^q_{2i} + alpha_i f^q_{2i-1} + gamma_i f^q_{2i+1},
//   top       x = D^{-1} f                     (the single remaining row),
//   backward  x^q_{2i} = x^{q+1}_i,
//             x^q_{2i+1} = D_{2i+1}^{-1} (f^q_{2i+1} - B_{2i+1} x^{q+1}_i - C_{2i+1} x^{q+1}_{i+1}),
// with a hardware cluster barrier between levels (no spin loops, no
// grid-wide dependency).  The wide levels keep their vectors in global memory
// (L2; chunks of rows staged into shared memory with cp.async); the levels of
// at most kRsSmall rows are finished by CTA 0 from its shared memory, their
// blocks copied in one batch, between __syncthreads.  The first level reads
// the FP64 right-hand side and writes the FP64 solution directly, converting
// as it goes.  The factors come from an FP32 cyclic reduction (or FP32 copies
// of an FP64 one).
#include <cuda_runtime.h>

#include "bt_bcr.cuh"
#include "bt_rsolve.h"

namespace bt {
namespace {

constexpr int kRsCtasMax = 16;   // non-portable cluster size, where it can be scheduled
constexpr int kRsCtasPortable = 8;
constexpr int kRsThreads = 512;

// Release/acquire at cluster scope orders every CTA's global-memory writes
// before the barrier with the other CTAs' reads after it (those reads go to
// L2: ld.global.cg).
__device__ __forceinline__ void cluster_barrier() {
    asm volatile(
        "barrier.cluster.arrive.release.aligned;\n"
        "barrier.cluster.wait.acquire.aligned;\n" ::
            : "memory");
}

__device__ __forceinline__ unsigned cluster_rank() {
    unsigned r;
    asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
    return r;
}
__device__ __forceinline__ unsigned cluster_size() {
    unsigned r;
    asm volatile("mov.u32 %0, %%cluster_nctarank;" : "=r"(r));
    return r;
}

// Exact FP32 -> FP64 by integer operations (FP32 subnormals become zero).
__device__ __forceinline__ double widen(float f) {
    const unsigned u = __float_as_uint(f);
    const unsigned sign = u & 0x80000000u, e = (u >> 23) & 0xffu, mant = u & 0x7fffffu;
    unsigned hi, lo = 0u;
    if (e == 0u) {
        hi = sign;
    } else if (e == 255u) {
        hi = sign | 0x7ff00000u | (mant >> 3) | (mant ? 0x80000u : 0u);
    } else {
        hi = sign | ((e + 896u) << 20) | (mant >> 3);
        lo = mant << 29;
    }
    return __hiloint2double((int)hi, (int)lo);
}

// Shared-memory staging: every level is processed in chunks of rows of this
// CTA's share; a chunk's blocks and vectors are copied with cp.async (16-byte
// copies through L2, past L1, every copy of the chunk in flight at once) and
// then used from shared memory.
__device__ __forceinline__ void rs_cp16(void* smem, const void* gmem) {
    const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(s), "l"(gmem) : "memory");
}
__device__ __forceinline__ void rs_cp_wait() {
    asm volatile("cp.async.commit_group;\ncp.async.wait_group 0;\n" ::: "memory");
}
__device__ __forceinline__ void stage_f4(float* dst, const float* src, long long n) {
    // n multiple of 4, both 16-byte aligned
    for (int e = threadIdx.x; e < (int)(n / 4); e += blockDim.x) rs_cp16(dst + 4 * e, src + 4 * e);
}
__device__ __forceinline__ void zero_f4(float* dst, long long n) {
    float4* d4 = reinterpret_cast<float4*>(dst);
    for (int e = threadIdx.x; e < (int)(n / 4); e += blockDim.x) d4[e] = make_float4(0.f, 0.f, 0.f, 0.f);
}

// The first level's right-hand side is the FP64 F0 and its solution the
// FP64 X0: they are converted where they are read and written (no separate
// conversion passes).  idx4 counts float4 units of the level vector.
__device__ __forceinline__ float4 get_f4(const RsolveArgs& a, int q, long long idx4) {
    if (q == 0) {
        const double2* s2 = reinterpret_cast<const double2*>(a.F0) + 2 * idx4;
        const double2 u = __ldcg(s2), w = __ldcg(s2 + 1);
        return make_float4(trunc_f32(u.x), trunc_f32(u.y), trunc_f32(w.x), trunc_f32(w.y));
    }
    return __ldcg(reinterpret_cast<const float4*>(a.f[q]) + idx4);
}
__device__ __forceinline__ void put_x4(const RsolveArgs& a, int q, long long idx4, float4 v) {
    if (q == 0) {
        double2* d2 = reinterpret_cast<double2*>(a.X0) + 2 * idx4;
        d2[0] = make_double2(widen(v.x), widen(v.y));
        d2[1] = make_double2(widen(v.z), widen(v.w));
    } else {
        reinterpret_cast<float4*>(a.x[q])[idx4] = v;
    }
}
__device__ __forceinline__ void put_x1(const RsolveArgs& a, int q, long long idx, float v) {
    if (q == 0) a.X0[idx] = widen(v);
    else a.x[q][idx] = v;
}
// dst <- f[q] entries [e0, e0 + n) (n and e0 multiples of 4): cp.async for the
// FP32 levels; the FP64 first level is loaded kRsUnroll float4 units per thread
// at a time (all loads issued before the converted values are stored).
constexpr int kRsUnroll = 4;
__device__ __forceinline__ void stage_fq(const RsolveArgs& a, int q, float* dst, long long e0, long long n) {
    if (q > 0) {
        stage_f4(dst, a.f[q] + e0, n);
        return;
    }
    float4* d4 = reinterpret_cast<float4*>(dst);
    const int n4 = (int)(n / 4), T = blockDim.x;
    for (int b = threadIdx.x; b < n4; b += kRsUnroll * T) {
        float4 v[kRsUnroll];
#pragma unroll
        for (int u = 0; u < kRsUnroll; ++u)
            if (b + u * T < n4) v[u] = get_f4(a, 0, e0 / 4 + b + u * T);
#pragma unroll
        for (int u = 0; u < kRsUnroll; ++u)
            if (b + u * T < n4) d4[b + u * T] = v[u];
    }
}

// dst <- the odd rows 2i + 1, i in [c0, c0 + n), of f^q (rows of E entries).
__device__ __forceinline__ void stage_odd_fq(const RsolveArgs& a, int q, float* dst, long long c0, int n, int E) {
    const int E4 = E / 4, n4 = n * E4, T = blockDim.x;
    if (q > 0) {
        for (int e = threadIdx.x; e < n4; e += T) {
            const int il = e / E4, w = e - il * E4;
            rs_cp16(dst + 4 * e, a.f[q] + (2 * (c0 + il) + 1) * E + 4 * w);
        }
        return;
    }
    float4* d4 = reinterpret_cast<float4*>(dst);
    for (int b = threadIdx.x; b < n4; b += kRsUnroll * T) {
        float4 v[kRsUnroll];
#pragma unroll
        for (int u = 0; u < kRsUnroll; ++u) {
            const int e = b + u * T;
            if (e < n4) {
                const int il = e / E4, w = e - il * E4;
                v[u] = get_f4(a, 0, (2 * (c0 + il) + 1) * E4 + w);
            }
        }
#pragma unroll
        for (int u = 0; u < kRsUnroll; ++u)
            if (b + u * T < n4) d4[b + u * T] = v[u];
    }
}

constexpr int kRsSmemFloats = 56 * 1024;   // 224 KB of shared memory per CTA
constexpr long long kRsSmall = 32;         // levels with at most this many rows run on CTA 0

// In shared memory an m x m block keeps its rows m + 4 floats apart: a row
// stays 16-byte aligned and read as float4 pieces, and the rows that the 8
// lanes of one shared-memory phase read fall in different banks.
__host__ __device__ constexpr int rs_row_stride(int m) { return m + 4; }
__host__ __device__ constexpr long long rs_block_floats(int m) { return (long long)m * rs_row_stride(m); }

// nblk consecutive m x m blocks from global memory into padded blocks.
template <int M>
__device__ __forceinline__ void stage_blocks(float* dst, const float* src, long long nblk) {
    constexpr int Q = M / 4, P = rs_row_stride(M);
    const int n = (int)nblk * M * Q;
    for (int e = threadIdx.x; e < n; e += blockDim.x) {
        const int row = e / Q, w = e - row * Q;   // row counts across the blocks
        rs_cp16(dst + row * P + 4 * w, src + (long long)row * M + 4 * w);
    }
}
// The blocks 2i + 1, i in [c0, c0 + nblk), of a level matrix.
template <int M>
__device__ __forceinline__ void stage_odd_blocks(float* dst, const float* src, long long c0, long long nblk) {
    constexpr int Q = M / 4, P = rs_row_stride(M), MM = M * M;
    const int n = (int)nblk * M * Q;
    for (int e = threadIdx.x; e < n; e += blockDim.x) {
        const int row = e / Q, w = e - row * Q, b = row / M, r = row - b * M;
        rs_cp16(dst + row * P + 4 * w, src + (2 * (c0 + b) + 1) * MM + r * M + 4 * w);
    }
}

// W consecutive floats (16-byte aligned for W == 4).
template <int W>
__device__ __forceinline__ void ldw(float (&v)[W], const float* p) {
    if constexpr (W == 4) {
        const float4 t = *reinterpret_cast<const float4*>(p);
        v[0] = t.x;
        v[1] = t.y;
        v[2] = t.z;
        v[3] = t.w;
    } else {
#pragma unroll
        for (int w = 0; w < W; ++w) v[w] = p[w];
    }
}
template <int W>
__device__ __forceinline__ void stw(float* p, const float (&v)[W]) {
    if constexpr (W == 4) {
        *reinterpret_cast<float4*>(p) = make_float4(v[0], v[1], v[2], v[3]);
    } else {
#pragma unroll
        for (int w = 0; w < W; ++w) p[w] = v[w];
    }
}
// s[w] +=(-=) sum_k A[k] X[k nr + w]: A one padded block row (float4 pieces),
// X the W columns of a block vector in shared memory.
template <int M, int W, bool NEG>
__device__ __forceinline__ void row_dot(float (&s)[W], const float* A, const float* X, int nr) {
#pragma unroll
    for (int kq = 0; kq < M / 4; ++kq) {
        const float4 a4 = *reinterpret_cast<const float4*>(A + 4 * kq);
        const float av[4] = {a4.x, a4.y, a4.z, a4.w};
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            float x[W];
            ldw<W>(x, X + (4 * kq + j) * nr);
#pragma unroll
            for (int w = 0; w < W; ++w) s[w] = fmaf(NEG ? -av[j] : av[j], x[w], s[w]);
        }
    }
}
// W entries of level q's solution (the FP64 X0 for q == 0).
template <int W>
__device__ __forceinline__ void put_xw(const RsolveArgs& a, int q, long long idx, const float (&v)[W]) {
    if constexpr (W == 4) {
        put_x4(a, q, idx / 4, make_float4(v[0], v[1], v[2], v[3]));
    } else {
#pragma unroll
        for (int w = 0; w < W; ++w) put_x1(a, q, idx + w, v[w]);
    }
}

// Forward step of level q for its kept rows [lo, hi): f^{q+1}_i = f_{2i} +
// alpha_i f_{2i-1} + gamma_i f_{2i+1}; chunks staged in shared memory.  A unit
// is (row, block-row entry, W columns).
template <int M, int W>
__device__ void rs_forward(const RsolveArgs& a, int q, long long lo, long long hi, float* sm) {
    constexpr int MM = M * M, P = rs_row_stride(M), MP = M * P;
    const int nr = a.nr, E = M * nr, EW = E / W;
    const long long K = a.K[q];
    const int CH = (a.chunk - E) / (2 * MP + 2 * E);
    for (long long c0 = lo; c0 < hi; c0 += CH) {
        const long long c1 = (c0 + CH < hi) ? c0 + CH : hi, n = c1 - c0;
        float* sal = sm;
        float* sga = sal + n * MP;
        float* sf = sga + n * MP;   // f rows 2 c0 - 1 .. 2 c1 - 1 (row 2 c0 - 1 at slot 0)
        stage_blocks<M>(sal, a.al[q] + c0 * MM, n);
        stage_blocks<M>(sga, a.ga[q] + c0 * MM, n);
        const long long f0 = 2 * c0 - 1, f1 = (2 * c1 < K) ? 2 * c1 : K;   // rows [f0, f1)
        if (f0 < 0) {
            zero_f4(sf, E);
            stage_fq(a, q, sf + E, 0, f1 * E);
        } else {
            stage_fq(a, q, sf, f0 * E, (f1 - f0) * E);
        }
        const long long nf = f1 - f0;
        if (nf < 2 * n + 1) zero_f4(sf + nf * E, (2 * n + 1 - nf) * E);
        rs_cp_wait();
        __syncthreads();
        for (int u = threadIdx.x; u < (int)n * EW; u += blockDim.x) {
            const int il = u / EW, e = (u - il * EW) * W, r = e / nr, c = e - r * nr;
            float s[W];
            ldw<W>(s, sf + (2 * il + 1) * E + e);
            row_dot<M, W, false>(s, sal + il * MP + r * P, sf + 2 * il * E + c, nr);
            row_dot<M, W, false>(s, sga + il * MP + r * P, sf + (2 * il + 2) * E + c, nr);
            stw<W>(a.f[q + 1] + (c0 + il) * E + e, s);
        }
        __syncthreads();
    }
}

// Back substitution of level q for the row pairs (2i, 2i+1), i in [lo, hi).
template <int M, int W>
__device__ void rs_backward(const RsolveArgs& a, int q, long long lo, long long hi, float* sm) {
    constexpr int MM = M * M, P = rs_row_stride(M), MP = M * P;
    const int nr = a.nr, E = M * nr, EW = E / W;
    const long long K = a.K[q], kept = (K + 1) / 2;
    const int CH = (a.chunk - E) / (3 * MP + 3 * E);
    for (long long c0 = lo; c0 < hi; c0 += CH) {
        const long long c1 = (c0 + CH < hi) ? c0 + CH : hi, n = c1 - c0;
        float* sB = sm;               // B of rows 2i+1
        float* sC = sB + n * MP;      // C of rows 2i+1
        float* sD = sC + n * MP;      // inverses of rows 2i+1
        float* sx = sD + n * MP;      // x^{q+1} rows c0 .. c1 (n + 1 rows)
        float* sf = sx + (n + 1) * E; // f rows 2i+1
        const long long nodd = (2 * c1 <= K) ? n : n - 1;   // row 2 c1 - 1 may not exist
        stage_odd_blocks<M>(sB, a.B[q], c0, nodd);
        stage_odd_blocks<M>(sC, a.C[q], c0, nodd);
        stage_blocks<M>(sD, a.Dinv[q] + c0 * MM, nodd);
        const long long xend = (c1 + 1 <= kept) ? c1 + 1 : kept;   // x^{q+1} rows [c0, xend)
        stage_f4(sx, a.x[q + 1] + c0 * E, (xend - c0) * E);
        stage_odd_fq(a, q, sf, c0, (int)nodd, E);
        if (xend - c0 < n + 1) zero_f4(sx + (xend - c0) * E, (n + 1 - (xend - c0)) * E);
        rs_cp_wait();
        __syncthreads();
        for (int u = threadIdx.x; u < (int)n * (E / 4); u += blockDim.x) {
            const int il = u / (E / 4);
            const int w = u - il * (E / 4);
            put_x4(a, q, (2 * (c0 + il)) * (E / 4) + w, reinterpret_cast<const float4*>(sx)[il * (E / 4) + w]);
        }
        // pass 1: t = f - B x_l - C x_r in place of f; pass 2: x = D^{-1} t
        for (int u = threadIdx.x; u < (int)nodd * EW; u += blockDim.x) {
            const int il = u / EW, e = (u - il * EW) * W, r = e / nr, c = e - r * nr;
            const long long rw = 2 * (c0 + il) + 1;
            float t[W];
            ldw<W>(t, sf + il * E + e);
            row_dot<M, W, true>(t, sB + il * MP + r * P, sx + il * E + c, nr);
            if (rw + 1 < K) row_dot<M, W, true>(t, sC + il * MP + r * P, sx + (il + 1) * E + c, nr);
            stw<W>(sf + il * E + e, t);
        }
        __syncthreads();
        for (int u = threadIdx.x; u < (int)nodd * EW; u += blockDim.x) {
            const int il = u / EW, e = (u - il * EW) * W, r = e / nr, c = e - r * nr;
            const long long rw = 2 * (c0 + il) + 1;
            float s[W];
#pragma unroll
            for (int w = 0; w < W; ++w) s[w] = 0.f;
            row_dot<M, W, false>(s, sD + il * MP + r * P, sf + il * E + c, nr);
            put_xw<W>(a, q, rw * E + e, s);
        }
        __syncthreads();
    }
}

// Shared-memory layout of the levels CTA 0 finishes alone, level q (K rows,
// (K+1)/2 kept, K/2 odd; the top level has only its inverse), blocks padded:
//   alpha, gamma [(K+1)/2] | D^{-1}, B, C of the odd rows [K/2] |
//   v [K][m][nr] (f^q, overwritten by x^q)
// and after the top level one scratch block of the odd rows' t vectors.  Every
// piece is a multiple of 4 floats (m >= 8), so each stays 16-byte aligned.
__host__ __device__ inline long long small_level_floats(long long K, int m, int nr, bool top) {
    const long long MP = rs_block_floats(m), E = (long long)m * nr;
    if (top) return MP + E;
    return 2 * ((K + 1) / 2) * MP + 3 * (K / 2) * MP + K * E;
}

// Levels [big, nlev) on one CTA, vectors and blocks in shared memory; W
// columns per unit (W = 4 when nr is a multiple of 4).
template <int M, int W>
__device__ void rs_small_levels(const RsolveArgs& a, float* S) {
    constexpr int P = rs_row_stride(M), MP = M * P;
    const int nr = a.nr, E = M * nr, EW = E / W, T = blockDim.x;
    const int top = a.nlev - 1, big = a.big;
    struct Lv {
        float *al, *ga, *di, *bb, *cc, *v;
    };
    auto lv = [&](int q) {
        const long long K = a.K[q], kept = (K + 1) / 2, odd = K / 2;
        Lv L;
        L.al = S + a.soff[q];
        if (q == top) {
            L.di = L.al;
            L.v = L.di + MP;
            L.ga = L.bb = L.cc = nullptr;
            return L;
        }
        L.ga = L.al + kept * MP;
        L.di = L.ga + kept * MP;
        L.bb = L.di + odd * MP;
        L.cc = L.bb + odd * MP;
        L.v = L.cc + odd * MP;
        return L;
    };
    float* tmp = S + a.soff[top + 1];
    // one batch of copies: every level's blocks and f^{big}
    for (int q = big; q <= top; ++q) {
        const Lv L = lv(q);
        if (q == top) {
            stage_blocks<M>(L.di, a.Dinv[q], 1);
            continue;
        }
        const long long K = a.K[q], kept = (K + 1) / 2, odd = K / 2;
        stage_blocks<M>(L.al, a.al[q], kept);
        stage_blocks<M>(L.ga, a.ga[q], kept);
        stage_blocks<M>(L.di, a.Dinv[q], odd);
        stage_odd_blocks<M>(L.bb, a.B[q], 0, odd);
        stage_odd_blocks<M>(L.cc, a.C[q], 0, odd);
    }
    stage_fq(a, big, lv(big).v, 0, a.K[big] * E);
    rs_cp_wait();
    __syncthreads();
    // forward: f^{q+1}_i = f_{2i} + alpha_i f_{2i-1} + gamma_i f_{2i+1}
    for (int q = big; q < top; ++q) {
        const Lv L = lv(q), N = lv(q + 1);
        const long long K = a.K[q], kept = (K + 1) / 2;
        for (int u = threadIdx.x; u < (int)kept * EW; u += T) {
            const int i = u / EW, e = (u - i * EW) * W, r = e / nr, c = e - r * nr;
            float s[W];
            ldw<W>(s, L.v + 2 * i * E + e);
            if (i > 0) row_dot<M, W, false>(s, L.al + i * MP + r * P, L.v + (2 * i - 1) * E + c, nr);
            if (2 * i + 1 < K) row_dot<M, W, false>(s, L.ga + i * MP + r * P, L.v + (2 * i + 1) * E + c, nr);
            stw<W>(N.v + i * E + e, s);
        }
        __syncthreads();
    }
    // top: x = D^{-1} f
    {
        const Lv L = lv(top);
        for (int u = threadIdx.x; u < EW; u += T) {
            const int e = u * W, r = e / nr, c = e - r * nr;
            float s[W];
#pragma unroll
            for (int w = 0; w < W; ++w) s[w] = 0.f;
            row_dot<M, W, false>(s, L.di + r * P, L.v + c, nr);
            stw<W>(tmp + e, s);
        }
        __syncthreads();
        for (int u = threadIdx.x; u < EW; u += T) {
            float x[W];
            ldw<W>(x, tmp + u * W);
            stw<W>(L.v + u * W, x);
        }
        __syncthreads();
    }
    // backward: x_{2i} = x^{q+1}_i; x_{2i+1} = D^{-1} (f_{2i+1} - B x_{2i} - C x_{2i+2})
    for (int q = top - 1; q >= big; --q) {
        const Lv L = lv(q), N = lv(q + 1);
        const long long K = a.K[q], kept = (K + 1) / 2, odd = K / 2;
        for (int u = threadIdx.x; u < (int)kept * EW; u += T) {
            const int i = u / EW, e = (u - i * EW) * W;
            float x[W];
            ldw<W>(x, N.v + i * E + e);
            stw<W>(L.v + 2 * i * E + e, x);
        }
        __syncthreads();
        for (int u = threadIdx.x; u < (int)odd * EW; u += T) {
            const int i = u / EW, e = (u - i * EW) * W, r = e / nr, c = e - r * nr;
            float t[W];
            ldw<W>(t, L.v + (2 * i + 1) * E + e);
            row_dot<M, W, true>(t, L.bb + i * MP + r * P, L.v + 2 * i * E + c, nr);
            if (2 * i + 2 < K) row_dot<M, W, true>(t, L.cc + i * MP + r * P, L.v + (2 * i + 2) * E + c, nr);
            stw<W>(tmp + i * E + e, t);
        }
        __syncthreads();
        for (int u = threadIdx.x; u < (int)odd * EW; u += T) {
            const int i = u / EW, e = (u - i * EW) * W, r = e / nr, c = e - r * nr;
            float s[W];
#pragma unroll
            for (int w = 0; w < W; ++w) s[w] = 0.f;
            row_dot<M, W, false>(s, L.di + i * MP + r * P, tmp + i * E + c, nr);
            stw<W>(L.v + (2 * i + 1) * E + e, s);
        }
        __syncthreads();
    }
    // x^{big} to its level vector (the FP64 solution when big == 0)
    {
        const float* v = lv(big).v;
        const long long n4 = a.K[big] * E / 4;
        for (long long u = threadIdx.x; u < n4; u += T) put_x4(a, big, u, reinterpret_cast<const float4*>(v)[u]);
    }
}

template <int M>
__global__ void __launch_bounds__(kRsThreads) k_rsolve_f32(const RsolveArgs a) {
    extern __shared__ __align__(16) float sm[];
    const int rank = (int)cluster_rank();
    const long long nct = (long long)cluster_size();
    const int big = a.big;
    const bool v4 = (a.nr & 3) == 0;
    // levels 0 .. big-1 run on the whole cluster, the rest on CTA 0 alone
    for (int q = 0; q < big; ++q) {
        const long long kept = (a.K[q] + 1) / 2, lo = kept * rank / nct, hi = kept * (rank + 1) / nct;
        if (v4) rs_forward<M, 4>(a, q, lo, hi, sm);
        else rs_forward<M, 1>(a, q, lo, hi, sm);
        cluster_barrier();
    }
    if (rank == 0) {
        if (v4) rs_small_levels<M, 4>(a, sm + a.chunk);
        else rs_small_levels<M, 1>(a, sm + a.chunk);
    }
    cluster_barrier();
    for (int q = big - 1; q >= 0; --q) {
        const long long kept = (a.K[q] + 1) / 2, lo = kept * rank / nct, hi = kept * (rank + 1) / nct;
        if (v4) rs_backward<M, 4>(a, q, lo, hi, sm);
        else rs_backward<M, 1>(a, q, lo, hi, sm);
        if (q > 0) cluster_barrier();
    }
}

// One grid row per segment (blockIdx.y), grid-stride within it.
__global__ void __launch_bounds__(256) k_cvt_f32(const CvtArgs a) {
    const int sgi = blockIdx.y;
    const double* s = a.src[sgi];
    float* d = a.dst[sgi];
    const long long n = a.n[sgi];
    for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (long long)gridDim.x * blockDim.x)
        d[e] = trunc_f32(s[e]);
}


// ---------------------------------------------------------------------------
// One-launch FP32 factorization of the reduced system by cyclic reduction
// (the refined paths, m = 8, 16): every level in one thread-block cluster,
// a cluster barrier between levels.  A kept row r = 2q of a level is handled
// by a pair of warps, one per side: side 0 inverts the left odd neighbour
// D_{r-1} and forms alpha_q = -B_r D_{r-1}^{-1}, alpha C_{r-1} and
// B'_q = alpha B_{r-1}; side 1 inverts D_{r+1} (stored as Dinv[q]) and forms
// gamma_q = -C_r D_{r+1}^{-1}, gamma B_{r+1} and C'_q = gamma C_{r+1}; side 0
// then writes D'_q = D_r + alpha C_{r-1} + gamma B_{r+1} (the pair meets at a
// named barrier).  In a warp, lane l holds columns [W h, W h + W) of row
// r = l mod m of a block (h = l / m, W = m^2 / 32).  The inverses are
// Gauss-Jordan eliminations with partial pivoting: the pivot of column k is
// found by a warp max-reduction over the rows not used yet, rows are not
// interchanged, the pivot row passes through shared memory and each row's
// multiplier through a shuffle.

constexpr int kRfThreads = 256;   // the cluster launch: 4 warp pairs per CTA, so that a CTA of
                                  // the level-0 forward solve still fits beside it on its SM
constexpr int kRfThreads0 = 64;   // the first level: one CTA (one warp pair) per kept row

template <int N>
__device__ __forceinline__ void rf_lds(float (&v)[N], const float* s) {
    if constexpr (N % 4 == 0) {
        const float4* p = reinterpret_cast<const float4*>(s);
#pragma unroll
        for (int u = 0; u < N / 4; ++u) {
            const float4 t = p[u];
            v[4 * u] = t.x;
            v[4 * u + 1] = t.y;
            v[4 * u + 2] = t.z;
            v[4 * u + 3] = t.w;
        }
    } else {
        const float2* p = reinterpret_cast<const float2*>(s);
#pragma unroll
        for (int u = 0; u < N / 2; ++u) {
            const float2 t = p[u];
            v[2 * u] = t.x;
            v[2 * u + 1] = t.y;
        }
    }
}
template <int N>
__device__ __forceinline__ void rf_sts(float* s, const float (&v)[N]) {
    if constexpr (N % 4 == 0) {
        float4* p = reinterpret_cast<float4*>(s);
#pragma unroll
        for (int u = 0; u < N / 4; ++u) p[u] = make_float4(v[4 * u], v[4 * u + 1], v[4 * u + 2], v[4 * u + 3]);
    } else {
        float2* p = reinterpret_cast<float2*>(s);
#pragma unroll
        for (int u = 0; u < N / 2; ++u) p[u] = make_float2(v[2 * u], v[2 * u + 1]);
    }
}
// N consecutive floats of global memory (L2), from FP32 or FP64 (truncated)
template <int N>
__device__ __forceinline__ void rf_ldg(float (&v)[N], const float* g) {
    if constexpr (N % 4 == 0) {
        const float4* p = reinterpret_cast<const float4*>(g);
#pragma unroll
        for (int u = 0; u < N / 4; ++u) {
            const float4 t = __ldcg(p + u);
            v[4 * u] = t.x;
            v[4 * u + 1] = t.y;
            v[4 * u + 2] = t.z;
            v[4 * u + 3] = t.w;
        }
    } else {
        const float2* p = reinterpret_cast<const float2*>(g);
#pragma unroll
        for (int u = 0; u < N / 2; ++u) {
            const float2 t = __ldcg(p + u);
            v[2 * u] = t.x;
            v[2 * u + 1] = t.y;
        }
    }
}
template <int N>
__device__ __forceinline__ void rf_ldg(float (&v)[N], const double* g) {
    const double2* p = reinterpret_cast<const double2*>(g);
#pragma unroll
    for (int u = 0; u < N / 2; ++u) {
        const double2 t = __ldcg(p + u);
        v[2 * u] = trunc_f32(t.x);
        v[2 * u + 1] = trunc_f32(t.y);
    }
}
template <int N>
__device__ __forceinline__ void rf_stg(float* g, const float (&v)[N]) { rf_sts<N>(g, v); }

// Gauss-Jordan inverse of an M x M block by one warp; lane (r, h) holds
// columns [W h, W h + W) of row r in a[] and of the identity in b[].  Column
// k's pivot is the unused row of largest magnitude (ties to the lowest row);
// no interchanges, so the lanes of the row that was column k's pivot end with
// their part of row k of the inverse in b[] and slot = k.  Returns false when
// a pivot column is zero (the result is then inf/nan).
template <int M>
__device__ __forceinline__ bool rf_inverse(float (&a)[M * M / 32], float (&b)[M * M / 32], int& slot, float* prow,
                                           int r, int h) {
    constexpr int W = M * M / 32;
    bool used = false, ok = true;
    slot = 0;
#pragma unroll
    for (int w = 0; w < W; ++w) b[w] = (W * h + w == r) ? 1.f : 0.f;
#pragma unroll
    for (int k = 0; k < M; ++k) {
        const int hk = k / W, kk = k % W;
        const float ak = a[kk];
        const unsigned key = (!used && h == hk) ? (__float_as_uint(ak) & 0x7fffffffu) + 1u : 0u;
        const unsigned kmax = __reduce_max_sync(0xffffffffu, key);
        const unsigned win = __ballot_sync(0xffffffffu, key == kmax);
        if (kmax <= 1u) ok = false;
        const int pr = (__ffs(win) - 1) % M;
        const float ark = __shfl_sync(0xffffffffu, ak, r + M * hk);   // this row's entry in column k
        const bool me = (r == pr);
        if (me) {
            used = true;
            slot = k;
            rf_sts<W>(prow + W * h, a);
            rf_sts<W>(prow + M + W * h, b);
        }
        __syncwarp();
        float pa[W], pb[W];
        rf_lds<W>(pa, prow + W * h);
        rf_lds<W>(pb, prow + M + W * h);
        const float inv = __frcp_rn(prow[k]);
        if (me) {
#pragma unroll
            for (int w = 0; w < W; ++w) {
                a[w] *= inv;
                b[w] *= inv;
            }
        } else {
            // paired FMAs (FFMA2), each component the scalar fmaf
            const float f = ark * inv;
            const float2 nf = make_float2(-f, -f);
#pragma unroll
            for (int w = 0; w < W; w += 2) {
                const float2 ta = __ffma2_rn(nf, make_float2(pa[w], pa[w + 1]), make_float2(a[w], a[w + 1]));
                const float2 tb = __ffma2_rn(nf, make_float2(pb[w], pb[w + 1]), make_float2(b[w], b[w + 1]));
                a[w] = ta.x;
                a[w + 1] = ta.y;
                b[w] = tb.x;
                b[w + 1] = tb.y;
            }
        }
        __syncwarp();
    }
    return ok;
}

// Columns [W h, W h + W) of row r of (sgn x S): x the full row in registers,
// S an M x M block in shared memory.
template <int M>
__device__ __forceinline__ void rf_row_part(float (&out)[M * M / 32], const float (&x)[M], const float* S, int h,
                                            float sgn) {
    constexpr int W = M * M / 32;
    float2 acc[W / 2];
#pragma unroll
    for (int w = 0; w < W / 2; ++w) acc[w] = make_float2(0.f, 0.f);
#pragma unroll
    for (int k = 0; k < M; ++k) {
        float srow[W];
        rf_lds<W>(srow, S + k * M + W * h);
        const float2 xk = make_float2(x[k], x[k]);
#pragma unroll
        for (int w = 0; w < W / 2; ++w) acc[w] = __ffma2_rn(xk, make_float2(srow[2 * w], srow[2 * w + 1]), acc[w]);
    }
#pragma unroll
    for (int w = 0; w < W / 2; ++w) {
        out[2 * w] = sgn * acc[w].x;
        out[2 * w + 1] = sgn * acc[w].y;
    }
}

template <int M, int NT>
constexpr size_t rf_smem_floats() {
    // per warp: inverse, two coupling blocks, the multiplier, pivot row; per pair: side 1's share of D'
    return (size_t)(NT / 32) * (4 * M * M + 2 * M) + (size_t)(NT / 64) * M * M;
}

__device__ __forceinline__ void pair_sync(int id) { asm volatile("bar.sync %0, 64;" ::"r"(id) : "memory"); }

// Levels [q0, q1).  CLUSTER: one thread-block cluster takes every level in
// turn (rows split over its CTAs, a cluster barrier between levels); else a
// plain grid takes the single level q0 (rows split over the CTAs) and also
// makes the FP32 copies of the first level's B and C.
template <int M, int NT, bool CLUSTER>
__global__ void __launch_bounds__(NT) k_rfactor_f32(const RfactorArgs a, int q0, int q1) {
    constexpr int W = M * M / 32;
    constexpr int MM = M * M;
    constexpr int NP = NT / 64;   // warp pairs per CTA
    extern __shared__ __align__(16) float sm[];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int r = lane % M, h = lane / M;
    const int side = warp & 1, pair = warp >> 1;
    float* ws = sm + warp * (4 * MM + 2 * M);
    float* Dv = ws;             // the inverse
    float* Y1 = ws + MM;        // the coupling blocks of the products
    float* Y2 = ws + 2 * MM;
    float* Mt = ws + 3 * MM;    // the multiplier
    float* prow = ws + 4 * MM;  // pivot row
    float* Ex = sm + (NT / 32) * (4 * MM + 2 * M) + pair * MM;   // side 1's share of D'
    const int rank = CLUSTER ? (int)cluster_rank() : (int)blockIdx.x;
    const long long nct = CLUSTER ? (long long)cluster_size() : (long long)gridDim.x;
    // the first level's side-1 tasks also leave FP32 copies of the odd rows'
    // B and C (all the solves read of that level's matrix)
    const bool copy0 = !CLUSTER && q0 == 0;
    for (int q = q0; q < q1; ++q) {
        const long long K = a.K[q];
        // row rr of block `which` (0 B, 1 D, 2 C) of this level: the whole row or this lane's part
        auto ldrow = [&](float (&v)[M], int which, long long rr) {
            if (q == 0) rf_ldg<M>(v, (which == 0 ? a.B0 : which == 1 ? a.D0 : a.C0) + rr * MM + r * M);
            else rf_ldg<M>(v, (which == 0 ? a.B[q] : which == 1 ? a.D[q] : a.C[q]) + rr * MM + r * M);
        };
        auto ldpart = [&](float (&v)[W], int which, long long rr) {
            if (q == 0) rf_ldg<W>(v, (which == 0 ? a.B0 : which == 1 ? a.D0 : a.C0) + rr * MM + r * M + W * h);
            else rf_ldg<W>(v, (which == 0 ? a.B[q] : which == 1 ? a.D[q] : a.C[q]) + rr * MM + r * M + W * h);
        };
        if (K == 1) {
            if (rank == 0 && warp == 0) {
                float x[W], inv[W];
                int slot;
                ldpart(x, 1, 0);
                if (!rf_inverse<M>(x, inv, slot, prow, r, h) && lane == 0)
                    report(a.status, ST_SINGULAR, a.level0 + q, -2, 0);
                rf_stg<W>(a.Dinv[q] + slot * M + W * h, inv);
            }
            break;
        }
        const long long kept = (K + 1) / 2;
        const long long lo = kept * rank / nct, hi = kept * (rank + 1) / nct;
        for (long long qq = lo + pair; qq < hi; qq += NP) {
            const long long rw = 2 * qq;
            const bool has = (side == 0) ? (qq >= 1) : (rw + 1 < K);
            const long long nb = (side == 0) ? rw - 1 : rw + 1;
            const bool far = (side == 0) ? (rw - 1 >= 1) : (rw + 2 < K);
            float* multo = ((side == 0) ? a.al[q] : a.ga[q]) + qq * MM + r * M + W * h;
            float* fout = ((side == 0) ? a.B[q + 1] : a.C[q + 1]) + qq * MM + r * M + W * h;
            float p1[W], p2[W], mlt[W];
#pragma unroll
            for (int w = 0; w < W; ++w) p1[w] = p2[w] = mlt[w] = 0.f;
            if (has) {
                // every block of the task is requested before the inverse starts
                float x[W], inv[W], c[M];
                int slot;
                ldpart(x, 1, nb);
                ldrow(c, side == 0 ? 0 : 2, rw);
                {
                    float y[W];
                    const long long o = nb * MM + r * M + W * h;
                    ldpart(y, side == 0 ? 2 : 0, nb);
                    rf_sts<W>(Y1 + r * M + W * h, y);
                    if (copy0 && q == 0 && side == 1) rf_stg<W>(a.B0f + o, y);
                    if (far) {
                        ldpart(y, side == 0 ? 0 : 2, nb);
                        rf_sts<W>(Y2 + r * M + W * h, y);
                    } else {
#pragma unroll
                        for (int w = 0; w < W; ++w) y[w] = 0.f;
                    }
                    if (copy0 && q == 0 && side == 1) rf_stg<W>(a.C0f + o, y);
                }
                if (!rf_inverse<M>(x, inv, slot, prow, r, h) && lane == 0)
                    report(a.status, ST_SINGULAR, a.level0 + q, -2, nb);
                rf_sts<W>(Dv + slot * M + W * h, inv);
                if (side == 1) rf_stg<W>(a.Dinv[q] + qq * MM + slot * M + W * h, inv);
                __syncwarp();
                rf_row_part<M>(mlt, c, Dv, h, -1.f);
                rf_sts<W>(Mt + r * M + W * h, mlt);
                __syncwarp();
                float mr[M];
                rf_lds<M>(mr, Mt + r * M);
                rf_row_part<M>(p1, mr, Y1, h, 1.f);
                if (far) rf_row_part<M>(p2, mr, Y2, h, 1.f);
            }
            rf_stg<W>(multo, mlt);
            rf_stg<W>(fout, p2);
            if (side == 1) rf_sts<W>(Ex + r * M + W * h, p1);
            pair_sync(1 + pair);
            if (side == 0) {
                float d[W], ex[W];
                ldpart(d, 1, rw);
                rf_lds<W>(ex, Ex + r * M + W * h);
#pragma unroll
                for (int w = 0; w < W; ++w) d[w] = (d[w] + p1[w]) + ex[w];
                rf_stg<W>(a.D[q + 1] + qq * MM + r * M + W * h, d);
            }
            pair_sync(1 + pair);
        }
        if (CLUSTER) cluster_barrier();
    }
}

}  // namespace

cudaError_t launch_cvt_f32(const CvtArgs& a, cudaStream_t s) {
    if (a.nseg <= 0) return cudaSuccess;
    long long mx = 0;
    for (int i = 0; i < a.nseg; ++i) mx = a.n[i] > mx ? a.n[i] : mx;
    long long bx = (mx + 255) / 256;
    if (bx < 1) bx = 1;
    if (bx > 256) bx = 256;
    k_cvt_f32<<<dim3((unsigned)bx, (unsigned)a.nseg), 256, 0, s>>>(a);
    return cudaGetLastError();
}

// The cluster size is chosen once per kernel (and device): 16 CTAs if the
// occupancy query places at least one such cluster, else 8.
template <typename K, typename Args>
static cudaError_t launch_cluster(K kernel, const Args& a, int threads, size_t smem, cudaStream_t s, int& ctas) {
    cudaLaunchConfig_t cfg = {};
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    cfg.blockDim = dim3(threads);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    if (ctas == 0) {
        cudaError_t e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        ctas = kRsCtasPortable;
        if (cudaFuncSetAttribute(kernel, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) == cudaSuccess) {
            cfg.gridDim = dim3(kRsCtasMax);
            at[0].val.clusterDim.x = kRsCtasMax;
            int n = 0;
            if (cudaOccupancyMaxActiveClusters(&n, kernel, &cfg) == cudaSuccess && n >= 1) ctas = kRsCtasMax;
        }
        cudaGetLastError();   // a refused query leaves no error behind
    }
    cfg.gridDim = dim3(ctas);
    at[0].val.clusterDim.x = ctas;
    return cudaLaunchKernelEx(&cfg, kernel, a);
}

template <typename K>
static cudaError_t launch_rs(K kernel, const RsolveArgs& a, cudaStream_t s, int& ctas) {
    return launch_cluster(kernel, a, kRsThreads, sizeof(float) * kRsSmemFloats, s, ctas);
}

// The first level (the widest) as a plain launch of one CTA per kept row, the
// others in one cluster launch.
template <int M>
static cudaError_t launch_rf(const RfactorArgs& a, cudaStream_t s, int& ctas) {
    const long long kept0 = (a.K[0] + 1) / 2;
    int q0 = 0;
    if (a.K[0] > 1) {
        const size_t smem0 = sizeof(float) * rf_smem_floats<M, kRfThreads0>();
        k_rfactor_f32<M, kRfThreads0, false><<<(unsigned)kept0, kRfThreads0, smem0, s>>>(a, 0, 1);
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
        q0 = 1;
    }
    if (q0 >= a.nlev) return cudaSuccess;
    const size_t smem = sizeof(float) * rf_smem_floats<M, kRfThreads>();
    auto kernel = k_rfactor_f32<M, kRfThreads, true>;
    cudaLaunchConfig_t cfg = {};
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    cfg.blockDim = dim3(kRfThreads);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    if (ctas == 0) {
        cudaError_t e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        ctas = kRsCtasPortable;
        if (cudaFuncSetAttribute(kernel, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) == cudaSuccess) {
            cfg.gridDim = dim3(kRsCtasMax);
            at[0].val.clusterDim.x = kRsCtasMax;
            int n = 0;
            if (cudaOccupancyMaxActiveClusters(&n, kernel, &cfg) == cudaSuccess && n >= 1) ctas = kRsCtasMax;
        }
        cudaGetLastError();
    }
    cfg.gridDim = dim3(ctas);
    at[0].val.clusterDim.x = ctas;
    return cudaLaunchKernelEx(&cfg, kernel, a, q0, a.nlev);
}

cudaError_t launch_rfactor_f32(const RfactorArgs& a, cudaStream_t s) {
    if (a.nlev < 1 || a.nlev > kRsMaxLevels) return cudaErrorInvalidValue;
    static int ctas[2] = {0, 0};
    switch (a.m) {
        case 8: return launch_rf<8>(a, s, ctas[0]);
        case 16: return launch_rf<16>(a, s, ctas[1]);
        default: return cudaErrorInvalidValue;
    }
}

// Split of the levels between the cluster and CTA 0 (the first level of at
// most kRsSmall rows, or a later one while CTA 0's share does not fit beside
// a chunk area of at least kRsMinChunk floats) and CTA 0's layout.
constexpr int kRsMinChunk = 16 * 1024;
static bool rs_layout(RsolveArgs& a) {
    const int top = a.nlev - 1, m = a.m, nr = a.nr;
    const long long MP = rs_block_floats(m), E = (long long)m * nr;
    long long minc = 3 * MP + 4 * E;
    if (minc < kRsMinChunk) minc = kRsMinChunk;
    int big = 0;
    while (big < top && a.K[big] > kRsSmall) ++big;
    for (;; ++big) {
        long long off = 0, tmpn = 0;
        for (int q = big; q <= top; ++q) {
            a.soff[q] = (int)off;
            off += small_level_floats(a.K[q], m, nr, q == top);
            const long long odd = (q == top) ? 1 : a.K[q] / 2;
            if (odd > tmpn) tmpn = odd;
        }
        a.soff[top + 1] = (int)off;
        off += tmpn * E;
        if (off + minc <= kRsSmemFloats) {
            a.big = big;
            a.chunk = (int)(kRsSmemFloats - off);
            return true;
        }
        if (big == top) return false;
    }
}

cudaError_t launch_rsolve_f32(const RsolveArgs& args, cudaStream_t s) {
    if (args.nlev < 1 || args.nlev > kRsMaxLevels || args.nr < 1 || args.nr > 32) return cudaErrorInvalidValue;
    RsolveArgs a = args;
    if (!rs_layout(a)) return cudaErrorInvalidValue;
    static int ctas[3] = {0, 0, 0};
    switch (a.m) {
        case 8: return launch_rs(k_rsolve_f32<8>, a, s, ctas[0]);
        case 16: return launch_rs(k_rsolve_f32<16>, a, s, ctas[1]);
        case 32: return launch_rs(k_rsolve_f32<32>, a, s, ctas[2]);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace bt
