// Refinement residuals r = f - A x of FP64 data in double-float arithmetic on
// the FP32 pipe (this GPU's FP64 pipe retires 2 FMA per clock per SM, its FP32
// pipe 128).  Method: every FP64 operand v is split exactly-in-range into
// v = v_hi + v_lo + O(2^-48 |v|) (v_hi: v truncated to FP32; v_lo: the
// remaining 29 mantissa bits rounded to FP32), the leading products
// a_hi x_hi are formed error-free (Dekker's TwoProduct with an FMA), summed
// with Knuth's TwoSum into a double-float accumulator, and the cross terms
// a_hi x_lo + a_lo x_hi plus all rounding errors are collected in a second
// FP32 accumulator (the compensated dot product "Dot2" of Ogita, Rump and
// Oishi, 2005).  Error per entry: of order sqrt(n) 2^-48 of
// sum_k |a_k||x_k| + |f| for n terms (the 48-bit operand splits and the FP32
// second accumulator; measured in an exact-arithmetic emulation at n = 48:
// mean 34, worst 218 units of 2^-53), against about sqrt(n) 2^-53 for FP64
// arithmetic -- the accuracy refinement to a 1e-10 forward error needs from
// its residual, at a fifth of the FP64 pipe's time.  The result is returned rounded to FP32 precision (stored as
// FP64): the correction solve that consumes it is FP32 anyway.
//
// Conversions between FP64 and FP32 are integer operations (no FP64 pipe).
// Operands with magnitude below 2^-74 keep only their FP32 part (relative
// error 2^-24 on those terms); the refined paths need entries inside the
// FP32 range in any case (their local factors are FP32).
#include <cuda_runtime.h>
#include <cstdint>

#include "bt_bcr.cuh"
#include "bt_misc.h"

namespace bt {
namespace {

// Exact FP32 -> FP64 by integer operations (FP32 subnormals become zero).
__device__ __forceinline__ double f32_to_f64(float f) {
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

__device__ __forceinline__ void two_sum(float a, float b, float& s, float& err) {
    s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    err = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}

// Compensated accumulator: value = s + l.
struct DF {
    float s, l;
    __device__ __forceinline__ void init(float2 v) {
        s = v.x;
        l = v.y;
    }
    // this -= a * x
    __device__ __forceinline__ void sub(float2 a, float2 x) {
        const float p = __fmul_rn(a.x, x.x);
        const float pe = fmaf(a.x, x.x, -p);
        float t;
        two_sum(s, -p, s, t);
        l = __fadd_rn(l, t);
        l = fmaf(-a.x, x.y, l);
        l = fmaf(-a.y, x.x, l);
        l = __fsub_rn(l, pe);
    }
    __device__ __forceinline__ void merge(const DF& o) {
        float t;
        two_sum(s, o.s, s, t);
        l = __fadd_rn(__fadd_rn(l, o.l), t);
    }
    __device__ __forceinline__ float value() const { return __fadd_rn(s, l); }
};

__device__ __forceinline__ unsigned long long abs_bits64(double v) {
    return (unsigned long long)__double_as_longlong(v) & 0x7fffffffffffffffull;
}
__device__ __forceinline__ unsigned long long umax_(unsigned long long a, unsigned long long b) {
    return a > b ? a : b;
}

// Largest of r, x, f over the block into slot (block mod kMaxSlots) of out
// (integer atomicMax); one call site, every thread of the block.
__device__ __forceinline__ void block_max3_df(unsigned long long r, unsigned long long x, unsigned long long f,
                                              unsigned long long* out) {
    __shared__ unsigned long long red[3][32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
        r = umax_(r, __shfl_xor_sync(0xffffffffu, r, off));
        x = umax_(x, __shfl_xor_sync(0xffffffffu, x, off));
        f = umax_(f, __shfl_xor_sync(0xffffffffu, f, off));
    }
    if (lane == 0) {
        red[0][warp] = r;
        red[1][warp] = x;
        red[2][warp] = f;
    }
    __syncthreads();
    if (threadIdx.x < 3) {
        unsigned long long v = 0ull;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) v = umax_(v, red[threadIdx.x][w]);
        atomicMax(out + 3 * (blockIdx.x % kMaxSlots) + threadIdx.x, v);
    }
}

constexpr int kDfThreads = 128;

__host__ __device__ inline int df_pair_shift(int nr);
// Block rows per CTA: enough (row, padded column pair) units for the 128 threads.
__host__ __device__ inline int df_rows_per_cta(int m, int nr) {
    const int units = m << df_pair_shift(nr);
    const int g = kDfThreads / units;
    return g < 1 ? 1 : g;
}

// Column pairs are padded to a power of two (cs = log2 of the padded count)
// so that the unit indices decompose by shifts; padded pairs are skipped.
__host__ __device__ inline int df_pair_shift(int nr) {
    const int ncp = (nr + 1) / 2;
    int sh = 0;
    while ((1 << sh) < ncp) ++sh;
    return sh;
}

// Stage x rows q0 .. q0 + nq - 1 of [rows][M][nr] (rows outside [0, rows)
// are zero) as double-float column pairs {hi_c, lo_c, hi_c+1, lo_c+1} at
// [q][k][pair] (padded pair count 2^cs); the magnitude maximum is taken over
// rows [own0, own1) only.
template <int M>
__device__ __forceinline__ unsigned long long stage_x(float4* sX, const double* X, long long rows, int nr, int cs,
                                                      long long q0, int nq, long long own0, long long own1) {
    const int ncp = (nr + 1) / 2;
    unsigned long long mx = 0ull;
    const int tot = (nq * M) << cs;
    for (int idx = threadIdx.x; idx < tot; idx += blockDim.x) {
        const int cp = idx & ((1 << cs) - 1), qk = idx >> cs, q = qk / M, k = qk % M;
        const long long j = q0 + q;
        float2 a = make_float2(0.f, 0.f), b = make_float2(0.f, 0.f);
        if (cp < ncp && j >= 0 && j < rows) {
            const double* src = X + (j * M + k) * nr + 2 * cp;
            const double v0 = src[0];
            a = split_f64(v0);
            unsigned long long m0 = abs_bits64(v0);
            if (2 * cp + 1 < nr) {
                const double v1 = src[1];
                b = split_f64(v1);
                m0 = umax_(m0, abs_bits64(v1));
            }
            if (j >= own0 && j < own1) mx = umax_(mx, m0);
        }
        sX[idx] = make_float4(a.x, a.y, b.x, b.y);
    }
    return mx;
}

// Block tridiagonal: CTA b takes block rows j0 = b G .. j0 + G - 1; thread
// unit (row j, block row entry r, column pair cp) accumulates
// f - B_j x_{j-1} - D_j x_j - C_j x_{j+1} for columns 2cp, 2cp+1, each over
// four compensated accumulators (term index mod 4; shorter chains for the
// FP32 second accumulator).
template <int M>
__global__ void __launch_bounds__(kDfThreads) k_resid_btri_df(long long N, int nr, int G,
                                                              const double* __restrict__ B,
                                                              const double* __restrict__ D,
                                                              const double* __restrict__ C,
                                                              const double* __restrict__ X,
                                                              const double* __restrict__ F, double* __restrict__ R,
                                                              unsigned long long* maxout) {
    extern __shared__ __align__(16) unsigned char smem[];
    constexpr int MM = M * M;
    const int ncp = (nr + 1) / 2, cs = df_pair_shift(nr), pcp = 1 << cs;
    float2* sA = reinterpret_cast<float2*>(smem);                      // [G][3][M][M]
    float4* sX = reinterpret_cast<float4*>(sA + (size_t)G * 3 * MM);   // [G + 2][M][pcp]
    const long long j0 = (long long)blockIdx.x * G;
    const int g = (int)((N - j0) < G ? (N - j0) : G);
    for (int idx = threadIdx.x; idx < g * 3 * MM; idx += blockDim.x) {
        const int gj = idx / (3 * MM), rem = idx % (3 * MM), which = rem / MM, e = rem % MM;
        const long long j = j0 + gj;
        const double* src = (which == 0) ? B : (which == 1 ? D : C);
        const bool present = (which == 1) || (which == 0 && j > 0) || (which == 2 && j + 1 < N);
        sA[idx] = present ? split_f64(src[j * MM + e]) : make_float2(0.f, 0.f);
    }
    unsigned long long mx = stage_x<M>(sX, X, N, nr, cs, j0 - 1, g + 2, j0, j0 + g);
    __syncthreads();
    unsigned long long mr = 0ull, mf = 0ull;
    for (int u = threadIdx.x; u < ((g * M) << cs); u += blockDim.x) {
        const int cp = u & (pcp - 1), gr = u >> cs, gj = gr / M, r = gr % M;
        if (cp >= ncp) continue;
        const long long row = (j0 + gj) * M + r;
        const int c0 = 2 * cp;
        const bool two = c0 + 1 < nr;
        const double f0 = F[row * nr + c0], f1 = two ? F[row * nr + c0 + 1] : 0.0;
        mf = umax_(mf, umax_(abs_bits64(f0), abs_bits64(f1)));
        DF a[4], b[4];
        a[0].init(split_f64(f0));
        b[0].init(split_f64(f1));
#pragma unroll
        for (int q = 1; q < 4; ++q) {
            a[q].init(make_float2(0.f, 0.f));
            b[q].init(make_float2(0.f, 0.f));
        }
#pragma unroll
        for (int blk = 0; blk < 3; ++blk) {
            const float2* Ar = sA + ((size_t)(gj * 3 + blk) * M + r) * M;
            const float4* xq = sX + (size_t)(gj + blk) * M * pcp + cp;
#pragma unroll
            for (int k = 0; k < M; ++k) {
                const float2 ak = Ar[k];
                const float4 xk = xq[k * pcp];
                a[k & 3].sub(ak, make_float2(xk.x, xk.y));
                b[k & 3].sub(ak, make_float2(xk.z, xk.w));
            }
        }
        DF& a0 = a[0];
        DF& b0 = b[0];
        a[0].merge(a[1]);
        a[2].merge(a[3]);
        a[0].merge(a[2]);
        b[0].merge(b[1]);
        b[2].merge(b[3]);
        b[0].merge(b[2]);
        const double r0 = f32_to_f64(a0.value());
        R[row * nr + c0] = r0;
        mr = umax_(mr, abs_bits64(r0));
        if (two) {
            const double r1 = f32_to_f64(b0.value());
            R[row * nr + c0 + 1] = r1;
            mr = umax_(mr, abs_bits64(r1));
        }
    }
    if (maxout) block_max3_df(mr, mx, mf, maxout);
}

// BABD (rows 0..N, boundary row first): row 0 is f_0 - B0 y_0 - B1 y_N, row
// j >= 1 is f_j - S_{j-1} y_{j-1} - R_{j-1} y_j.  x slots: the rows
// j0 - 1 .. j0 + g - 1, and (CTA 0 only) y_N after them.
template <int M>
__global__ void __launch_bounds__(kDfThreads) k_resid_babd_df(long long N, int nr, int G,
                                                              const double* __restrict__ S,
                                                              const double* __restrict__ Rm,
                                                              const double* __restrict__ B0,
                                                              const double* __restrict__ B1,
                                                              const double* __restrict__ Y,
                                                              const double* __restrict__ F,
                                                              double* __restrict__ Rout, unsigned long long* maxout) {
    extern __shared__ __align__(16) unsigned char smem[];
    constexpr int MM = M * M;
    const int ncp = (nr + 1) / 2, cs = df_pair_shift(nr), pcp = 1 << cs;
    float2* sA = reinterpret_cast<float2*>(smem);                      // [G][2][M][M]
    float4* sX = reinterpret_cast<float4*>(sA + (size_t)G * 2 * MM);   // [G + 2][M][pcp]
    const long long rows = N + 1;
    const long long j0 = (long long)blockIdx.x * G;
    const int g = (int)((rows - j0) < G ? (rows - j0) : G);
    for (int idx = threadIdx.x; idx < g * 2 * MM; idx += blockDim.x) {
        const int gj = idx / (2 * MM), rem = idx % (2 * MM), which = rem / MM, e = rem % MM;
        const long long j = j0 + gj;
        const double v = (j == 0) ? (which == 0 ? B0[e] : B1[e]) : (which == 0 ? S : Rm)[(j - 1) * MM + e];
        sA[idx] = split_f64(v);
    }
    unsigned long long mx = stage_x<M>(sX, Y, rows, nr, cs, j0 - 1, g + 1, j0, j0 + g);
    if (j0 == 0) stage_x<M>(sX + (size_t)(g + 1) * M * pcp, Y, rows, nr, cs, N, 1, 0, 0);
    __syncthreads();
    unsigned long long mr = 0ull, mf = 0ull;
    for (int u = threadIdx.x; u < ((g * M) << cs); u += blockDim.x) {
        const int cp = u & (pcp - 1), gr = u >> cs, gj = gr / M, r = gr % M;
        if (cp >= ncp) continue;
        const long long j = j0 + gj;
        const long long row = j * M + r;
        const int c0 = 2 * cp;
        const bool two = c0 + 1 < nr;
        const double f0 = F[row * nr + c0], f1 = two ? F[row * nr + c0 + 1] : 0.0;
        mf = umax_(mf, umax_(abs_bits64(f0), abs_bits64(f1)));
        DF a[4], b[4];
        a[0].init(split_f64(f0));
        b[0].init(split_f64(f1));
#pragma unroll
        for (int q = 1; q < 4; ++q) {
            a[q].init(make_float2(0.f, 0.f));
            b[q].init(make_float2(0.f, 0.f));
        }
#pragma unroll
        for (int blk = 0; blk < 2; ++blk) {
            const float2* Ar = sA + ((size_t)(gj * 2 + blk) * M + r) * M;
            const int slot = (j == 0) ? (blk == 0 ? 1 : g + 1) : gj + blk;
            const float4* xq = sX + (size_t)slot * M * pcp + cp;
#pragma unroll
            for (int k = 0; k < M; ++k) {
                const float2 ak = Ar[k];
                const float4 xk = xq[k * pcp];
                a[k & 3].sub(ak, make_float2(xk.x, xk.y));
                b[k & 3].sub(ak, make_float2(xk.z, xk.w));
            }
        }
        DF& a0 = a[0];
        DF& b0 = b[0];
        a[0].merge(a[1]);
        a[2].merge(a[3]);
        a[0].merge(a[2]);
        b[0].merge(b[1]);
        b[2].merge(b[3]);
        b[0].merge(b[2]);
        const double r0 = f32_to_f64(a0.value());
        Rout[row * nr + c0] = r0;
        mr = umax_(mr, abs_bits64(r0));
        if (two) {
            const double r1 = f32_to_f64(b0.value());
            Rout[row * nr + c0 + 1] = r1;
            mr = umax_(mr, abs_bits64(r1));
        }
    }
    if (maxout) block_max3_df(mr, mx, mf, maxout);
}

__device__ __forceinline__ void df_cp16(void* smem, const void* gmem) {
    const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(sa), "l"(gmem) : "memory");
}
__device__ __forceinline__ void df_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N>
__device__ __forceinline__ void df_wait() {
    asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory");
}

// Persistent, pipelined form of k_resid_btri_df: each CTA strides over tiles
// of G block rows; the FP64 blocks, x rows and f rows of the next tile are
// copied into a second shared buffer (cp.async, 16-byte pieces) while the
// current tile is split into double-float form and reduced.  Needs 16-byte
// aligned arrays and an even number of entries per block row of x (m nr).
template <int M>
__global__ void __launch_bounds__(kDfThreads) k_resid_btri_df2(long long N, int nr, int G, long long ntiles,
                                                               const double* __restrict__ B,
                                                               const double* __restrict__ D,
                                                               const double* __restrict__ C,
                                                               const double* __restrict__ X,
                                                               const double* __restrict__ F, double* __restrict__ R,
                                                               unsigned long long* maxout) {
    extern __shared__ __align__(16) unsigned char smem[];
    constexpr int MM = M * M;
    const int ncp = (nr + 1) / 2, cs = df_pair_shift(nr), pcp = 1 << cs;
    const int V = M * nr;                                  // doubles per block row of x or f
    const int nA = G * 3 * MM, nX = (G + 2) * V, nF = G * V;
    const int nraw = nA + nX + nF;
    double* raw0 = reinterpret_cast<double*>(smem);
    double* raw1 = raw0 + nraw;
    float2* sA = reinterpret_cast<float2*>(raw1 + nraw);   // [G][3][M][M]
    float4* sX = reinterpret_cast<float4*>(sA + nA);       // [G + 2][M][pcp]
    const double* arr[3] = {B, D, C};
    auto issue = [&](long long t, double* raw) {
        if (t < ntiles) {
            const long long j0 = t * G;
            const int g = (int)((N - j0) < G ? (N - j0) : G);
            for (int w = 0; w < 3; ++w) {
                const double* src = arr[w] + j0 * MM;
                double* dst = raw + w * G * MM;
                for (int c = threadIdx.x; c < g * MM / 2; c += blockDim.x) df_cp16(dst + 2 * c, src + 2 * c);
            }
            const long long lo = (j0 - 1 > 0) ? j0 - 1 : 0, hi = (j0 + g + 1 < N) ? j0 + g + 1 : N;
            double* dx = raw + nA + (lo - (j0 - 1)) * V;
            const double* sx = X + lo * V;
            for (int c = threadIdx.x; c < (int)(hi - lo) * V / 2; c += blockDim.x) df_cp16(dx + 2 * c, sx + 2 * c);
            const double* sf = F + j0 * V;
            for (int c = threadIdx.x; c < g * V / 2; c += blockDim.x) df_cp16(raw + nA + nX + 2 * c, sf + 2 * c);
        }
        df_commit();
    };
    unsigned long long mr = 0ull, mx = 0ull, mf = 0ull;
    int buf = 0;
    issue(blockIdx.x, raw0);
    for (long long t = blockIdx.x; t < ntiles; t += gridDim.x, buf ^= 1) {
        double* raw = buf ? raw1 : raw0;
        issue(t + gridDim.x, buf ? raw0 : raw1);
        df_wait<1>();
        __syncthreads();
        const long long j0 = t * G;
        const int g = (int)((N - j0) < G ? (N - j0) : G);
        for (int idx = threadIdx.x; idx < g * 3 * MM; idx += blockDim.x) {
            const int gj = idx / (3 * MM), rem = idx % (3 * MM), w = rem / MM, e = rem % MM;
            const long long j = j0 + gj;
            const bool present = (w == 1) || (w == 0 && j > 0) || (w == 2 && j + 1 < N);
            sA[idx] = present ? split_f64(raw[w * G * MM + gj * MM + e]) : make_float2(0.f, 0.f);
        }
        for (int idx = threadIdx.x; idx < ((g + 2) * M) << cs; idx += blockDim.x) {
            const int cp = idx & (pcp - 1), qk = idx >> cs, q = qk / M, k = qk % M;
            const long long row = j0 - 1 + q;
            float2 a = make_float2(0.f, 0.f), b = make_float2(0.f, 0.f);
            if (cp < ncp && row >= 0 && row < N) {
                const double* src = raw + nA + q * V + k * nr + 2 * cp;
                const double v0 = src[0];
                a = split_f64(v0);
                unsigned long long m0 = abs_bits64(v0);
                if (2 * cp + 1 < nr) {
                    const double v1 = src[1];
                    b = split_f64(v1);
                    m0 = umax_(m0, abs_bits64(v1));
                }
                if (q >= 1 && q <= g) mx = umax_(mx, m0);
            }
            sX[idx] = make_float4(a.x, a.y, b.x, b.y);
        }
        __syncthreads();
        const double* rf = raw + nA + nX;
        for (int u = threadIdx.x; u < ((g * M) << cs); u += blockDim.x) {
            const int cp = u & (pcp - 1), gr = u >> cs, gj = gr / M, r = gr % M;
            if (cp >= ncp) continue;
            const long long row = (j0 + gj) * M + r;
            const int c0 = 2 * cp;
            const bool two = c0 + 1 < nr;
            const double f0 = rf[(gj * M + r) * nr + c0], f1 = two ? rf[(gj * M + r) * nr + c0 + 1] : 0.0;
            mf = umax_(mf, umax_(abs_bits64(f0), abs_bits64(f1)));
            DF a[4], b[4];
            a[0].init(split_f64(f0));
            b[0].init(split_f64(f1));
#pragma unroll
            for (int qq = 1; qq < 4; ++qq) {
                a[qq].init(make_float2(0.f, 0.f));
                b[qq].init(make_float2(0.f, 0.f));
            }
#pragma unroll
            for (int blk = 0; blk < 3; ++blk) {
                const float2* Ar = sA + ((gj * 3 + blk) * M + r) * M;
                const float4* xq = sX + (gj + blk) * M * pcp + cp;
#pragma unroll
                for (int k = 0; k < M; ++k) {
                    const float2 ak = Ar[k];
                    const float4 xk = xq[k * pcp];
                    a[k & 3].sub(ak, make_float2(xk.x, xk.y));
                    b[k & 3].sub(ak, make_float2(xk.z, xk.w));
                }
            }
            a[0].merge(a[1]);
            a[2].merge(a[3]);
            a[0].merge(a[2]);
            b[0].merge(b[1]);
            b[2].merge(b[3]);
            b[0].merge(b[2]);
            const double r0 = f32_to_f64(a[0].value());
            R[row * nr + c0] = r0;
            mr = umax_(mr, abs_bits64(r0));
            if (two) {
                const double r1 = f32_to_f64(b[0].value());
                R[row * nr + c0 + 1] = r1;
                mr = umax_(mr, abs_bits64(r1));
            }
        }
        __syncthreads();
    }
    df_wait<0>();
    if (maxout) block_max3_df(mr, mx, mf, maxout);
}

// Variant of k_resid_btri_df2 for matrices kept as FP32 pairs (hi, lo) by the
// warp-per-partition factorization (float2 [3][N][M][M]): the pairs are
// copied straight into a double-buffered shared array, so only x and f are
// split per call.
template <int M>
__global__ void __launch_bounds__(kDfThreads) k_resid_btri_dfs(long long N, int nr, int G, long long ntiles,
                                                               const float2* __restrict__ As,
                                                               const double* __restrict__ X,
                                                               const double* __restrict__ F, double* __restrict__ R,
                                                               unsigned long long* maxout) {
    extern __shared__ __align__(16) unsigned char smem[];
    constexpr int MM = M * M;
    const int ncp = (nr + 1) / 2, cs = df_pair_shift(nr), pcp = 1 << cs;
    const int V = M * nr;
    const int nA = G * 3 * MM, nX = (G + 2) * V, nF = G * V;
    float2* sA0 = reinterpret_cast<float2*>(smem);          // [G][3][M][M], two buffers
    float2* sA1 = sA0 + nA;
    double* raw0 = reinterpret_cast<double*>(sA1 + nA);     // x, f rows, two buffers
    double* raw1 = raw0 + (nX + nF);
    float4* sX = reinterpret_cast<float4*>(raw1 + (nX + nF));   // [G + 2][M][pcp]
    auto issue = [&](long long t, float2* sA, double* raw) {
        if (t < ntiles) {
            const long long j0 = t * G;
            const int g = (int)((N - j0) < G ? (N - j0) : G);
            for (int c = threadIdx.x; c < g * 3 * (MM / 2); c += blockDim.x) {
                const int blk = c / (MM / 2), piece = c % (MM / 2), gj = blk / 3, w = blk % 3;
                df_cp16(sA + (gj * 3 + w) * MM + 2 * piece, As + (w * N + j0 + gj) * MM + 2 * piece);
            }
            const long long lo = (j0 - 1 > 0) ? j0 - 1 : 0, hi = (j0 + g + 1 < N) ? j0 + g + 1 : N;
            double* dx = raw + (lo - (j0 - 1)) * V;
            const double* sx = X + lo * V;
            for (int c = threadIdx.x; c < (int)(hi - lo) * V / 2; c += blockDim.x) df_cp16(dx + 2 * c, sx + 2 * c);
            const double* sf = F + j0 * V;
            for (int c = threadIdx.x; c < g * V / 2; c += blockDim.x) df_cp16(raw + nX + 2 * c, sf + 2 * c);
        }
        df_commit();
    };
    unsigned long long mr = 0ull, mx = 0ull, mf = 0ull;
    int buf = 0;
    issue(blockIdx.x, sA0, raw0);
    for (long long t = blockIdx.x; t < ntiles; t += gridDim.x, buf ^= 1) {
        float2* sA = buf ? sA1 : sA0;
        double* raw = buf ? raw1 : raw0;
        issue(t + gridDim.x, buf ? sA0 : sA1, buf ? raw0 : raw1);
        df_wait<1>();
        __syncthreads();
        const long long j0 = t * G;
        const int g = (int)((N - j0) < G ? (N - j0) : G);
        for (int idx = threadIdx.x; idx < ((g + 2) * M) << cs; idx += blockDim.x) {
            const int cp = idx & (pcp - 1), qk = idx >> cs, q = qk / M, k = qk % M;
            const long long row = j0 - 1 + q;
            float2 a = make_float2(0.f, 0.f), b = make_float2(0.f, 0.f);
            if (cp < ncp && row >= 0 && row < N) {
                const double* src = raw + q * V + k * nr + 2 * cp;
                const double v0 = src[0];
                a = split_f64(v0);
                unsigned long long m0 = abs_bits64(v0);
                if (2 * cp + 1 < nr) {
                    const double v1 = src[1];
                    b = split_f64(v1);
                    m0 = umax_(m0, abs_bits64(v1));
                }
                if (q >= 1 && q <= g) mx = umax_(mx, m0);
            }
            sX[idx] = make_float4(a.x, a.y, b.x, b.y);
        }
        __syncthreads();
        const double* rf = raw + nX;
        for (int u = threadIdx.x; u < ((g * M) << cs); u += blockDim.x) {
            const int cp = u & (pcp - 1), gr = u >> cs, gj = gr / M, r = gr % M;
            if (cp >= ncp) continue;
            const long long row = (j0 + gj) * M + r;
            const int c0 = 2 * cp;
            const bool two = c0 + 1 < nr;
            const double f0 = rf[(gj * M + r) * nr + c0], f1 = two ? rf[(gj * M + r) * nr + c0 + 1] : 0.0;
            mf = umax_(mf, umax_(abs_bits64(f0), abs_bits64(f1)));
            DF a[4], b[4];
            a[0].init(split_f64(f0));
            b[0].init(split_f64(f1));
#pragma unroll
            for (int qq = 1; qq < 4; ++qq) {
                a[qq].init(make_float2(0.f, 0.f));
                b[qq].init(make_float2(0.f, 0.f));
            }
#pragma unroll
            for (int blk = 0; blk < 3; ++blk) {
                const float2* Ar = sA + ((gj * 3 + blk) * M + r) * M;
                const float4* xq = sX + (gj + blk) * M * pcp + cp;
#pragma unroll
                for (int k = 0; k < M; ++k) {
                    const float2 ak = Ar[k];
                    const float4 xk = xq[k * pcp];
                    a[k & 3].sub(ak, make_float2(xk.x, xk.y));
                    b[k & 3].sub(ak, make_float2(xk.z, xk.w));
                }
            }
            a[0].merge(a[1]);
            a[2].merge(a[3]);
            a[0].merge(a[2]);
            b[0].merge(b[1]);
            b[2].merge(b[3]);
            b[0].merge(b[2]);
            const double r0 = f32_to_f64(a[0].value());
            R[row * nr + c0] = r0;
            mr = umax_(mr, abs_bits64(r0));
            if (two) {
                const double r1 = f32_to_f64(b[0].value());
                R[row * nr + c0 + 1] = r1;
                mr = umax_(mr, abs_bits64(r1));
            }
        }
        __syncthreads();
    }
    df_wait<0>();
    if (maxout) block_max3_df(mr, mx, mf, maxout);
}

template <typename K>
cudaError_t launch_df(K kernel, size_t smem, long long ctas, cudaStream_t s) {
    if (smem > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
    }
    (void)ctas;
    return cudaSuccess;
}

}  // namespace

static size_t resid_dfs_smem(int m, int nr, int G) {
    const int pcp = 1 << df_pair_shift(nr), V = m * nr;
    const size_t nA = (size_t)G * 3 * m * m, nX = (size_t)(G + 2) * V, nF = (size_t)G * V;
    return 2 * nA * sizeof(float2) + 2 * (nX + nF) * sizeof(double) + (size_t)(G + 2) * m * pcp * sizeof(float4);
}

cudaError_t launch_resid_btri_dfs(long long N, int m, int nr, const float2* As, const double* X, const double* F,
                                  double* R, cudaStream_t s, unsigned long long* maxout) {
    if (N <= 0) return cudaSuccess;
    if (m != 16 || ((uintptr_t)As | (uintptr_t)X | (uintptr_t)F) & 15u) return cudaErrorInvalidValue;
    int G = df_rows_per_cta(m, nr);
    while (G > 1 && resid_dfs_smem(m, nr, G) > 180 * 1024) --G;
    const long long ntiles = (N + G - 1) / G;
    const size_t smem = resid_dfs_smem(m, nr, G);
    int dev = 0, sms = 148;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    long long per_sm = (long long)(200 * 1024) / (long long)smem;
    if (per_sm > 8) per_sm = 8;
    if (per_sm < 1) per_sm = 1;
    long long grid = per_sm * sms;
    if (grid > ntiles) grid = ntiles;
    cudaError_t e = launch_df(k_resid_btri_dfs<16>, smem, grid, s);
    if (e != cudaSuccess) return e;
    k_resid_btri_dfs<16><<<(unsigned)grid, kDfThreads, smem, s>>>(N, nr, G, ntiles, As, X, F, R, maxout);
    return cudaGetLastError();
}

size_t resid_df_smem(int kind, int m, int nr) {
    const int G = df_rows_per_cta(m, nr), pcp = 1 << df_pair_shift(nr);
    const size_t a = (size_t)G * (kind == 0 ? 3 : 2) * m * m * sizeof(float2);
    return a + (size_t)(G + 2) * m * pcp * sizeof(float4);
}

static size_t resid_df2_smem(int m, int nr, int G) {
    const int pcp = 1 << df_pair_shift(nr), V = m * nr;
    const size_t nA = (size_t)G * 3 * m * m, nX = (size_t)(G + 2) * V, nF = (size_t)G * V;
    return 2 * (nA + nX + nF) * sizeof(double) + nA * sizeof(float2) + (size_t)(G + 2) * m * pcp * sizeof(float4);
}

cudaError_t launch_resid_btri_df(long long N, int m, int nr, const double* B, const double* D, const double* C,
                                 const double* X, const double* F, double* R, cudaStream_t s,
                                 unsigned long long* maxout) {
    if (N <= 0) return cudaSuccess;
    const uintptr_t al = (uintptr_t)B | (uintptr_t)D | (uintptr_t)C | (uintptr_t)X | (uintptr_t)F;
    if (m >= 8 && ((m * nr) % 2) == 0 && (al & 15u) == 0) {
        // persistent pipelined kernel: a few CTAs per SM stride over tiles
        // block rows per tile: enough units for the threads, within 180 KB of shared memory
        int G = df_rows_per_cta(m, nr);
        while (G > 1 && resid_df2_smem(m, nr, G) > 180 * 1024) --G;
        const long long ntiles = (N + G - 1) / G;
        const size_t smem = resid_df2_smem(m, nr, G);
        int dev = 0, sms = 148;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        long long per_sm = (long long)(200 * 1024) / (long long)smem;
        if (per_sm > 8) per_sm = 8;
        if (per_sm < 1) per_sm = 1;
        long long grid = per_sm * sms;
        if (grid > ntiles) grid = ntiles;
        cudaError_t e = cudaSuccess;
        switch (m) {
            case 8:
                e = launch_df(k_resid_btri_df2<8>, smem, grid, s);
                if (e == cudaSuccess)
                    k_resid_btri_df2<8><<<(unsigned)grid, kDfThreads, smem, s>>>(N, nr, G, ntiles, B, D, C, X, F, R, maxout);
                break;
            case 16:
                e = launch_df(k_resid_btri_df2<16>, smem, grid, s);
                if (e == cudaSuccess)
                    k_resid_btri_df2<16><<<(unsigned)grid, kDfThreads, smem, s>>>(N, nr, G, ntiles, B, D, C, X, F, R, maxout);
                break;
            default:
                e = launch_df(k_resid_btri_df2<32>, smem, grid, s);
                if (e == cudaSuccess)
                    k_resid_btri_df2<32><<<(unsigned)grid, kDfThreads, smem, s>>>(N, nr, G, ntiles, B, D, C, X, F, R, maxout);
                break;
        }
        if (e != cudaSuccess) return e;
        return cudaGetLastError();
    }
    const int G = df_rows_per_cta(m, nr);
    const long long ctas = (N + G - 1) / G;
    const size_t smem = resid_df_smem(0, m, nr);
    cudaError_t e = cudaSuccess;
#define BT_DF_CASE(MV)                                                                                    \
    case MV:                                                                                              \
        e = launch_df(k_resid_btri_df<MV>, smem, ctas, s);                                                \
        if (e == cudaSuccess)                                                                             \
            k_resid_btri_df<MV><<<(unsigned)ctas, kDfThreads, smem, s>>>(N, nr, G, B, D, C, X, F, R, maxout); \
        break;
    switch (m) {
        BT_DF_CASE(1)
        BT_DF_CASE(2)
        BT_DF_CASE(4)
        BT_DF_CASE(8)
        BT_DF_CASE(16)
        BT_DF_CASE(32)
        default: return cudaErrorInvalidValue;
    }
#undef BT_DF_CASE
    if (e != cudaSuccess) return e;
    return cudaGetLastError();
}

cudaError_t launch_resid_babd_df(long long N, int m, int nr, const double* S, const double* Rm, const double* B0,
                                 const double* B1, const double* Y, const double* F, double* Rout, cudaStream_t s,
                                 unsigned long long* maxout) {
    const int G = df_rows_per_cta(m, nr);
    const long long ctas = (N + 1 + G - 1) / G;
    const size_t smem = resid_df_smem(1, m, nr);
    cudaError_t e = cudaSuccess;
#define BT_DF_CASE(MV)                                                                                      \
    case MV:                                                                                                \
        e = launch_df(k_resid_babd_df<MV>, smem, ctas, s);                                                  \
        if (e == cudaSuccess)                                                                               \
            k_resid_babd_df<MV><<<(unsigned)ctas, kDfThreads, smem, s>>>(N, nr, G, S, Rm, B0, B1, Y, F, Rout, \
                                                                          maxout);                          \
        break;
    switch (m) {
        BT_DF_CASE(1)
        BT_DF_CASE(2)
        BT_DF_CASE(4)
        BT_DF_CASE(8)
        BT_DF_CASE(16)
        BT_DF_CASE(32)
        default: return cudaErrorInvalidValue;
    }
#undef BT_DF_CASE
    if (e != cudaSuccess) return e;
    return cudaGetLastError();
}

}  // namespace bt
