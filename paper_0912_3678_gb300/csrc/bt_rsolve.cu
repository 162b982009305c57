// Solve of the reduced system (Eq. (redmatr)) by block cyclic reduction in one
// launch, for the refined paths: the FP64 cyclic-reduction factors (computed
// by k_bcr_factor, Sec. 2 cyclic-reduction variant) are applied as FP32
// copies, inside the FP32 correction solve that the FP64 refinement
// corrects.  One thread-block cluster of kRsCtas CTAs runs every level:
//   forward   f^{q+1}_i = f^q_{2i} + alpha_i f^q_{2i-1} + gamma_i f^q_{2i+1},
//   top       x = D^{-1} f                     (the single remaining row),
//   backward  x^q_{2i} = x^{q+1}_i,
//             x^q_{2i+1} = D_{2i+1}^{-1} (f^q_{2i+1} - B_{2i+1} x^{q+1}_i - C_{2i+1} x^{q+1}_{i+1}),
// with a hardware cluster barrier between levels (no spin loops, no
// grid-wide dependency); levels with at most kRsCluster rows are finished by
// one CTA between __syncthreads.  The level vectors live in global memory (L2)
// and are read past L1 (ld.global.cg).
#include <cuda_runtime.h>

#include "bt_bcr.cuh"
#include "bt_rsolve.h"

namespace bt {
namespace {

constexpr int kRsCtas = 8;
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
// CTA's share; a chunk's blocks and vectors arrive in one round of coalesced
// 16-byte loads (L2, past L1) and are then used from shared memory.
__device__ __forceinline__ void stage_f4(float* dst, const float* src, long long n) {
    // n multiple of 4, both 16-byte aligned
    const float4* s4 = reinterpret_cast<const float4*>(src);
    float4* d4 = reinterpret_cast<float4*>(dst);
    for (int e = threadIdx.x; e < (int)(n / 4); e += blockDim.x) d4[e] = __ldcg(s4 + e);
}
__device__ __forceinline__ void zero_f4(float* dst, long long n) {
    float4* d4 = reinterpret_cast<float4*>(dst);
    for (int e = threadIdx.x; e < (int)(n / 4); e += blockDim.x) d4[e] = make_float4(0.f, 0.f, 0.f, 0.f);
}

constexpr int kRsSmemFloats = 24 * 1024;   // 96 KB of shared memory per CTA
constexpr long long kRsCluster = 64;       // levels with more rows run on the whole cluster

// Forward step of level q for its kept rows [lo, hi): f^{q+1}_i = f_{2i} +
// alpha_i f_{2i-1} + gamma_i f_{2i+1}; chunks staged in shared memory.  With
// nr a multiple of 4 a unit is (row, block-row entry, 4 columns).
template <int M>
__device__ void rs_forward(const RsolveArgs& a, int q, long long lo, long long hi, float* sm) {
    constexpr int MM = M * M;
    const int nr = a.nr, E = M * nr;
    const long long K = a.K[q];
    const int CH = (kRsSmemFloats - E) / (2 * MM + 2 * E);
    const bool v4 = (nr & 3) == 0;
    for (long long c0 = lo; c0 < hi; c0 += CH) {
        const long long c1 = (c0 + CH < hi) ? c0 + CH : hi, n = c1 - c0;
        float* sal = sm;
        float* sga = sal + n * MM;
        float* sf = sga + n * MM;   // f rows 2 c0 - 1 .. 2 c1 - 1 (row 2 c0 - 1 at slot 0)
        stage_f4(sal, a.al[q] + c0 * MM, n * MM);
        stage_f4(sga, a.ga[q] + c0 * MM, n * MM);
        const long long f0 = 2 * c0 - 1, f1 = (2 * c1 < K) ? 2 * c1 : K;   // rows [f0, f1)
        if (f0 < 0) {
            zero_f4(sf, E);
            stage_f4(sf + E, a.f[q], f1 * E);
        } else {
            stage_f4(sf, a.f[q] + f0 * E, (f1 - f0) * E);
        }
        const long long nf = f1 - f0;
        if (nf < 2 * n + 1) zero_f4(sf + nf * E, (2 * n + 1 - nf) * E);
        __syncthreads();
        if (v4) {
            const int E4 = E / 4, n4 = nr / 4;
            const float4* sf4 = reinterpret_cast<const float4*>(sf);
            for (int u = threadIdx.x; u < (int)n * E4; u += blockDim.x) {
                const int il = u / E4, e4 = u - il * E4, r = e4 / n4, c4 = e4 - r * n4;
                const float* A = sal + il * MM + r * M;
                const float* G = sga + il * MM + r * M;
                const float4* vl = sf4 + (2 * il) * E4 + c4;
                const float4* vr = sf4 + (2 * il + 2) * E4 + c4;
                float4 s = sf4[(2 * il + 1) * E4 + e4];
#pragma unroll
                for (int k = 0; k < M; ++k) {
                    const float ak = A[k], gk = G[k];
                    const float4 x0 = vl[k * n4], x1 = vr[k * n4];
                    s.x = fmaf(ak, x0.x, fmaf(gk, x1.x, s.x));
                    s.y = fmaf(ak, x0.y, fmaf(gk, x1.y, s.y));
                    s.z = fmaf(ak, x0.z, fmaf(gk, x1.z, s.z));
                    s.w = fmaf(ak, x0.w, fmaf(gk, x1.w, s.w));
                }
                reinterpret_cast<float4*>(a.f[q + 1])[(c0 + il) * E4 + e4] = s;
            }
        } else {
            for (int u = threadIdx.x; u < (int)n * E; u += blockDim.x) {
                const int il = u / E, el = u - il * E, r = el / nr, c = el - r * nr;
                const float* A = sal + il * MM + r * M;
                const float* G = sga + il * MM + r * M;
                const float* vl = sf + (2 * il) * E + c;
                const float* vr = sf + (2 * il + 2) * E + c;
                float s0 = sf[(2 * il + 1) * E + el], s1 = 0.f;
#pragma unroll
                for (int k = 0; k < M; ++k) {
                    s0 = fmaf(A[k], vl[k * nr], s0);
                    s1 = fmaf(G[k], vr[k * nr], s1);
                }
                a.f[q + 1][(c0 + il) * E + el] = s0 + s1;
            }
        }
        __syncthreads();
    }
}

// Back substitution of level q for the row pairs (2i, 2i+1), i in [lo, hi).
template <int M>
__device__ void rs_backward(const RsolveArgs& a, int q, long long lo, long long hi, float* sm) {
    constexpr int MM = M * M;
    const int nr = a.nr, E = M * nr;
    const long long K = a.K[q], kept = (K + 1) / 2;
    const int CH = (kRsSmemFloats - E) / (3 * MM + 3 * E);
    const bool v4 = (nr & 3) == 0;
    for (long long c0 = lo; c0 < hi; c0 += CH) {
        const long long c1 = (c0 + CH < hi) ? c0 + CH : hi, n = c1 - c0;
        float* sB = sm;               // B of rows 2i+1
        float* sC = sB + n * MM;      // C of rows 2i+1
        float* sD = sC + n * MM;      // inverses of rows 2i+1
        float* sx = sD + n * MM;      // x^{q+1} rows c0 .. c1 (n + 1 rows)
        float* sf = sx + (n + 1) * E; // f rows 2i+1
        const long long nodd = (2 * c1 <= K) ? n : n - 1;   // row 2 c1 - 1 may not exist
        for (int e = threadIdx.x; e < (int)nodd * (MM / 4); e += blockDim.x) {
            const int il = e / (MM / 4), w = e % (MM / 4);
            const long long rw = 2 * (c0 + il) + 1;
            reinterpret_cast<float4*>(sB)[e] = __ldcg(reinterpret_cast<const float4*>(a.B[q] + rw * MM) + w);
            reinterpret_cast<float4*>(sC)[e] = __ldcg(reinterpret_cast<const float4*>(a.C[q] + rw * MM) + w);
        }
        for (int e = threadIdx.x; e < (int)nodd * (E / 4); e += blockDim.x) {
            const int il = e / (E / 4), w = e - il * (E / 4);
            reinterpret_cast<float4*>(sf)[e] =
                __ldcg(reinterpret_cast<const float4*>(a.f[q] + (2 * (c0 + il) + 1) * E) + w);
        }
        stage_f4(sD, a.Dinv[q] + c0 * MM, nodd * MM);
        const long long xend = (c1 + 1 <= kept) ? c1 + 1 : kept;   // x^{q+1} rows [c0, xend)
        stage_f4(sx, a.x[q + 1] + c0 * E, (xend - c0) * E);
        if (xend - c0 < n + 1) zero_f4(sx + (xend - c0) * E, (n + 1 - (xend - c0)) * E);
        __syncthreads();
        for (int u = threadIdx.x; u < (int)n * (E / 4); u += blockDim.x) {
            const int il = u / (E / 4);
            const int w = u - il * (E / 4);
            reinterpret_cast<float4*>(a.x[q])[(2 * (c0 + il)) * (E / 4) + w] = reinterpret_cast<const float4*>(sx)[il * (E / 4) + w];
        }
        // pass 1: t = f - B x_l - C x_r in place of f; pass 2: x = D^{-1} t
        if (v4) {
            const int n4 = nr / 4, E4 = E / 4;
            const float4* sx4 = reinterpret_cast<const float4*>(sx);
            float4* sf4 = reinterpret_cast<float4*>(sf);
            for (int u = threadIdx.x; u < (int)nodd * E4; u += blockDim.x) {
                const int il = u / E4, e4 = u - il * E4, r = e4 / n4, c4 = e4 - r * n4;
                const long long rw = 2 * (c0 + il) + 1;
                const float rm = (rw + 1 < K) ? 1.f : 0.f;
                const float* Bo = sB + il * MM + r * M;
                const float* Co = sC + il * MM + r * M;
                float4 t = sf4[il * E4 + e4];
#pragma unroll
                for (int k = 0; k < M; ++k) {
                    const float b = Bo[k], cc = Co[k] * rm;
                    const float4 xl = sx4[il * E4 + k * n4 + c4], xr = sx4[(il + 1) * E4 + k * n4 + c4];
                    t.x = fmaf(-b, xl.x, fmaf(-cc, xr.x, t.x));
                    t.y = fmaf(-b, xl.y, fmaf(-cc, xr.y, t.y));
                    t.z = fmaf(-b, xl.z, fmaf(-cc, xr.z, t.z));
                    t.w = fmaf(-b, xl.w, fmaf(-cc, xr.w, t.w));
                }
                sf4[il * E4 + e4] = t;
            }
            __syncthreads();
            for (int u = threadIdx.x; u < (int)nodd * E4; u += blockDim.x) {
                const int il = u / E4, e4 = u - il * E4, r = e4 / n4, c4 = e4 - r * n4;
                const long long rw = 2 * (c0 + il) + 1;
                const float* Di = sD + il * MM + r * M;
                float4 x = make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
                for (int k = 0; k < M; ++k) {
                    const float d = Di[k];
                    const float4 t = sf4[il * E4 + k * n4 + c4];
                    x.x = fmaf(d, t.x, x.x);
                    x.y = fmaf(d, t.y, x.y);
                    x.z = fmaf(d, t.z, x.z);
                    x.w = fmaf(d, t.w, x.w);
                }
                reinterpret_cast<float4*>(a.x[q])[rw * E4 + e4] = x;
            }
        } else {
            for (int u = threadIdx.x; u < (int)nodd * E; u += blockDim.x) {
                const int il = u / E, el = u - il * E, r = el / nr, c = el - r * nr;
                const long long rw = 2 * (c0 + il) + 1;
                const float rm = (rw + 1 < K) ? 1.f : 0.f;
                const float* Bo = sB + il * MM + r * M;
                const float* Co = sC + il * MM + r * M;
                const float* xl = sx + il * E + c;
                const float* xr = sx + (il + 1) * E + c;
                float s0 = sf[il * E + el], s1 = 0.f;
#pragma unroll
                for (int k = 0; k < M; ++k) {
                    s0 = fmaf(-Bo[k], xl[k * nr], s0);
                    s1 = fmaf(-Co[k] * rm, xr[k * nr], s1);
                }
                sf[il * E + el] = s0 + s1;
            }
            __syncthreads();
            for (int u = threadIdx.x; u < (int)nodd * E; u += blockDim.x) {
                const int il = u / E, el = u - il * E, r = el / nr, c = el - r * nr;
                const long long rw = 2 * (c0 + il) + 1;
                const float* Di = sD + il * MM + r * M;
                float s0 = 0.f, s1 = 0.f;
#pragma unroll
                for (int k = 0; k < M; k += 2) {
                    s0 = fmaf(Di[k], sf[il * E + k * nr + c], s0);
                    s1 = fmaf(Di[k + 1], sf[il * E + (k + 1) * nr + c], s1);
                }
                a.x[q][rw * E + el] = s0 + s1;
            }
        }
        __syncthreads();
    }
}

template <int M>
__global__ void __cluster_dims__(kRsCtas, 1, 1) __launch_bounds__(kRsThreads) k_rsolve_f32(const RsolveArgs a) {
    extern __shared__ __align__(16) float sm[];
    const int nr = a.nr;
    const int E = M * nr;   // multiple of 4 (M >= 8)
    const int rank = (int)cluster_rank();
    const long long T = (long long)kRsCtas * kRsThreads;
    const long long t0 = (long long)rank * kRsThreads + threadIdx.x;
    const int top = a.nlev - 1;
    // levels 0 .. big-1 run on the whole cluster, the rest on CTA 0 alone
    int big = 0;
    while (big < top && a.K[big] > kRsCluster) ++big;
    for (long long e = t0; e < a.K[0] * E; e += T) a.f[0][e] = trunc_f32(a.F0[e]);
    cluster_barrier();
    for (int q = 0; q < big; ++q) {
        const long long kept = (a.K[q] + 1) / 2;
        rs_forward<M>(a, q, kept * rank / kRsCtas, kept * (rank + 1) / kRsCtas, sm);
        cluster_barrier();
    }
    if (rank == 0) {
        for (int q = big; q < top; ++q) {
            rs_forward<M>(a, q, 0, (a.K[q] + 1) / 2, sm);   // ends with __syncthreads
        }
        const float* Di = a.Dinv[top];
        const float* f = a.f[top];
        for (int u = threadIdx.x; u < E; u += blockDim.x) {
            const int r = u / nr, c = u % nr;
            float s = 0.f;
#pragma unroll
            for (int k = 0; k < M; ++k) s = fmaf(Di[r * M + k], __ldcg(f + k * nr + c), s);
            a.x[top][u] = s;
        }
        __syncthreads();
        for (int q = top - 1; q >= big; --q) rs_backward<M>(a, q, 0, (a.K[q] + 1) / 2, sm);
    }
    cluster_barrier();
    for (int q = big - 1; q >= 0; --q) {
        const long long kept = (a.K[q] + 1) / 2;
        rs_backward<M>(a, q, kept * rank / kRsCtas, kept * (rank + 1) / kRsCtas, sm);
        cluster_barrier();
    }
    for (long long e = t0; e < a.K[0] * E; e += T) a.X0[e] = widen(__ldcg(a.x[0] + e));
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

template <typename K>
static cudaError_t launch_rs(K kernel, const RsolveArgs& a, cudaStream_t s) {
    const size_t smem = sizeof(float) * kRsSmemFloats;
    cudaError_t e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    kernel<<<kRsCtas, kRsThreads, smem, s>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_rsolve_f32(const RsolveArgs& a, cudaStream_t s) {
    if (a.nlev < 1 || a.nlev > kRsMaxLevels || a.nr < 1 || a.nr > 32) return cudaErrorInvalidValue;
    switch (a.m) {
        case 8: return launch_rs(k_rsolve_f32<8>, a, s);
        case 16: return launch_rs(k_rsolve_f32<16>, a, s);
        case 32: return launch_rs(k_rsolve_f32<32>, a, s);
        default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

}  // namespace bt
