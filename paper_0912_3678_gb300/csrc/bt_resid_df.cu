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
#include <cuda_bf16.h>
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

// The compensated accumulator on the paired FP32 instructions of this GPU
// (FMUL2, FFMA2, FADD2: two FP32 operations per issued instruction, each
// component rounded as its scalar form).  The two components hold the sums
// over the even and the odd k of one entry, merged at the end; each component
// takes the steps of DF.sub in the same order.  The matrix entries come
// negated, (-a_hi, -a_hi+1) and (-a_lo, -a_lo+1) for k, k + 1, so every step
// adds: a difference x - y is the fused y * (-1) + x (exact product, one
// rounding) and no operand is negated in flight.
__device__ __forceinline__ float2 sub2(float2 x, float2 y) { return __ffma2_rn(y, make_float2(-1.f, -1.f), x); }
struct DFk {
    float2 s, l;
    __device__ __forceinline__ void init(float s0, float l0) {
        s = make_float2(s0, 0.f);
        l = make_float2(l0, 0.f);
    }
    __device__ __forceinline__ void zero() { s = l = make_float2(0.f, 0.f); }
    // this += (-a) x for k and k + 1: na = (-a_hi), nl = (-a_lo), xh / xl the
    // high and low parts of x_k, x_k+1
    __device__ __forceinline__ void add(float2 na, float2 nl, float2 xh, float2 xl) {
        const float2 q = __fmul2_rn(na, xh);                                          // -p
        const float2 qe = __ffma2_rn(na, xh, sub2(make_float2(0.f, 0.f), q));         // -(a_hi x_hi - p)
        const float2 s1 = __fadd2_rn(s, q);
        const float2 bb = sub2(s1, s);
        const float2 t = __fadd2_rn(sub2(s, sub2(s1, bb)), sub2(q, bb));
        s = s1;
        l = __fadd2_rn(l, t);
        l = __ffma2_rn(na, xl, l);
        l = __ffma2_rn(nl, xh, l);
        l = __fadd2_rn(l, qe);
    }
    __device__ __forceinline__ void merge(const DFk& o) {
        const float2 s1 = __fadd2_rn(s, o.s);
        const float2 bb = sub2(s1, s);
        const float2 t = __fadd2_rn(sub2(s, sub2(s1, bb)), sub2(o.s, bb));
        s = s1;
        l = __fadd2_rn(__fadd2_rn(l, o.l), t);
    }
    // the two components' sums merged, rounded to FP32
    __device__ __forceinline__ float value() const {
        float sv, t;
        two_sum(s.x, s.y, sv, t);
        return __fadd_rn(sv, __fadd_rn(__fadd_rn(l.x, l.y), t));
    }
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

// Variant of k_resid_btri_df2 for the matrix kept by the warp-per-partition
// factorization as negated FP32 pairs by column pairs, float4 [3][N][M][M/2]
// of (-hi_k, -hi_k+1, -lo_k, -lo_k+1) for even k: the blocks are copied
// straight into a double-buffered shared array, so only x and f are split per
// call (into the same k-pair form).  A thread takes one row entry of two
// right-hand-side columns, each column in two k-pair accumulators.
template <int M>
__global__ void __launch_bounds__(kDfThreads) k_resid_btri_dfs(long long N, int nr, int G, long long ntiles,
                                                               const float2* __restrict__ As,
                                                               const double* __restrict__ X,
                                                               const double* __restrict__ F, double* __restrict__ R,
                                                               unsigned long long* maxout) {
    extern __shared__ __align__(16) unsigned char smem[];
    constexpr int MM = M * M, KP = M / 2;
    const int ncp = (nr + 1) / 2, cs = df_pair_shift(nr), pcp = 1 << cs;
    const int V = M * nr;
    const int nA = G * 3 * MM, nX = (G + 2) * V, nF = G * V;
    float2* sA0 = reinterpret_cast<float2*>(smem);          // [G][3][M][M], two buffers
    float2* sA1 = sA0 + nA;
    double* raw0 = reinterpret_cast<double*>(sA1 + nA);     // x, f rows, two buffers
    double* raw1 = raw0 + (nX + nF);
    float4* sX = reinterpret_cast<float4*>(raw1 + (nX + nF));   // [G + 2][KP][2 pcp] k-pair form
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
        // x_k, x_k+1 of columns 2 cp, 2 cp + 1 -> two k-pair entries of sX
        for (int idx = threadIdx.x; idx < ((g + 2) * KP) << cs; idx += blockDim.x) {
            const int cp = idx & (pcp - 1), qk = idx >> cs, q = qk / KP, kp = qk % KP;
            const long long row = j0 - 1 + q;
            float2 a0 = make_float2(0.f, 0.f), a1 = a0, b0 = a0, b1 = a0;   // (column, k) = (0,0), (0,1), (1,0), (1,1)
            if (cp < ncp && row >= 0 && row < N) {
                const double* src = raw + q * V + 2 * kp * nr + 2 * cp;
                const double v00 = src[0], v01 = src[nr];
                a0 = split_f64(v00);
                a1 = split_f64(v01);
                unsigned long long m0 = umax_(abs_bits64(v00), abs_bits64(v01));
                if (2 * cp + 1 < nr) {
                    const double v10 = src[1], v11 = src[nr + 1];
                    b0 = split_f64(v10);
                    b1 = split_f64(v11);
                    m0 = umax_(m0, umax_(abs_bits64(v10), abs_bits64(v11)));
                }
                if (q >= 1 && q <= g) mx = umax_(mx, m0);
            }
            float4* d = sX + (q * KP + kp) * 2 * pcp + 2 * cp;
            d[0] = make_float4(a0.x, a1.x, a0.y, a1.y);
            d[1] = make_float4(b0.x, b1.x, b0.y, b1.y);
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
            DFk a[2], b[2];   // columns c0 (a) and c0 + 1 (b), two accumulators each
            {
                const float2 s0 = split_f64(f0), s1 = split_f64(f1);
                a[0].init(s0.x, s0.y);
                b[0].init(s1.x, s1.y);
                a[1].zero();
                b[1].zero();
            }
#pragma unroll
            for (int blk = 0; blk < 3; ++blk) {
                const float4* Ar = reinterpret_cast<const float4*>(sA + ((gj * 3 + blk) * M + r) * M);
                const float4* xq = sX + (gj + blk) * KP * 2 * pcp + 2 * cp;
#pragma unroll
                for (int kp = 0; kp < KP; ++kp) {
                    const float4 ak = Ar[kp];
                    const float4 x0 = xq[kp * 2 * pcp], x1 = xq[kp * 2 * pcp + 1];
                    const float2 na = make_float2(ak.x, ak.y), nl = make_float2(ak.z, ak.w);
                    a[kp & 1].add(na, nl, make_float2(x0.x, x0.y), make_float2(x0.z, x0.w));
                    b[kp & 1].add(na, nl, make_float2(x1.x, x1.y), make_float2(x1.z, x1.w));
                }
            }
            a[0].merge(a[1]);
            b[0].merge(b[1]);
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
    // the kernels also hold static shared memory (the maxima reduction), so the
    // dynamic limit is raised whenever the dynamic part comes near 48 KB
    if (smem > 40 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
    }
    (void)ctas;
    return cudaSuccess;
}


// ---------------------------------------------------------------------------
// The same residual (block tridiagonal, m = 16, up to 8 right-hand sides)
// with the products on the tensor cores, by the error-free splitting of
// Ozaki, Ogita, Oishi and Rump (2012): every row i of [B_j D_j C_j] is scaled
// by 2^(E_i) (E_i the exponent of the row's largest entry) and written as
// seven signed 8-bit digits, a_ik = sum_p s_ikp 2^(E_i - 7 - 8p) (the value
// truncated 56 bits below the row maximum); every column n of the window
// [x_{j-1}; x_j; x_{j+1}] likewise with its own exponent F_n.  A digit is an
// integer of magnitude below 256, exact in BF16; a product of two digits is
// below 2^16 and exact in FP32, and a sum of 48 of them (one block row) below
// 2^21.6.  The products of digit planes p and q are accumulated per weight
// t = p + q by BF16 mma.sync m16n8k16 tiles with FP32 accumulation: exact
// for t <= 5 (at most 3 planes pairs per accumulator, below 2^24), and for
// t = 6, 7 rounded at 2^-54 of (row maximum x column maximum).  Planes with
// t >= 8 are dropped (below 2^-54 of the same).  The weighted sum
// sum_t acc_t 2^(56 - 8t) is formed in double-float arithmetic (Knuth's
// TwoSum), scaled by 2^(E_i + F_n - 70), subtracted from f in double-float
// and rounded to FP32 (stored as FP64), as the other double-float residuals.
// Error: about 2^-49 of |A|_max |x|_max per entry, below the refinement's
// stopping threshold 4(3m+1) 2^-53 (normwise) by a factor 100.
//
// One warp per block row; lane (g, t) = (lane / 4, lane % 4) holds the MMA
// fragments: rows g and g + 8, columns 2t, 2t+1, 2t+8, 2t+9 of each 16 x 16
// block of A, rows 2t, 2t+1, 2t+8, 2t+9 of column g of each x block.
constexpr int kOzThreads = 256;

// exponent field (biased) of |v|, 0 for zero and subnormals
__device__ __forceinline__ int oz_expo(double v) { return (__double2hiint(v) >> 20) & 0x7ff; }

// The seven 8-bit digits of |v| below 2^(eb - 1022) (eb: biased exponent of
// the scale, eb >= the exponent of v), as floats with the sign of v, most
// significant first.
__device__ __forceinline__ void oz_digits(double v, int eb, float (&d)[7]) {
    const unsigned hw = (unsigned)__double2hiint(v), lw = (unsigned)__double2loint(v);
    const int ef = (int)((hw >> 20) & 0x7ffu);
    const unsigned sgn = hw & 0x80000000u;
    unsigned long long I = 0ull;
    if (ef != 0 && ef != 0x7ff) {
        const unsigned long long Mv = ((unsigned long long)((hw & 0xfffffu) | 0x100000u) << 32) | lw;
        const int sh = ef - eb + 3;   // v = M 2^(ef - 1075) = I 2^(eb - 1023 - 55)
        if (sh >= 0) I = Mv << sh;
        else if (sh > -64) I = Mv >> (-sh);
    }
    const unsigned ih = (unsigned)(I >> 32), il = (unsigned)I;
#pragma unroll
    for (int p = 0; p < 7; ++p) {
        const int bpos = 6 - p;   // byte of I holding digit p
        const unsigned b = (bpos >= 4) ? ((ih >> (8 * (bpos - 4))) & 0xffu) : ((il >> (8 * bpos)) & 0xffu);
        const float f = __fsub_rn(__uint_as_float(0x4b000000u | b), 8388608.f);
        d[p] = __uint_as_float(__float_as_uint(f) | sgn);
    }
}

__device__ __forceinline__ unsigned oz_pack(float lo, float hi) {
    const __nv_bfloat162 v = __floats2bfloat162_rn(lo, hi);
    return *reinterpret_cast<const unsigned*>(&v);
}

__device__ __forceinline__ void oz_mma(float (&c)[4], const unsigned (&a)[4], unsigned b0, unsigned b1) {
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
        "{%0,%1,%2,%3};"
        : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

// Tiles of kOzRows block rows (one per warp): A blocks (rows padded to 18
// doubles against bank conflicts), the x rows of the window and f, staged by
// cp.async, two tiles in flight.
constexpr int kOzRows = kOzThreads / 32;
constexpr int kOzLd = 18;                       // padded row of a 16 x 16 block
constexpr int kOzBlk = 16 * kOzLd;              // doubles per staged block
__host__ __device__ constexpr int oz_stage_doubles(int nr) {
    return kOzRows * 3 * kOzBlk + (kOzRows + 2) * 16 * nr + kOzRows * 16 * nr;
}

__device__ __forceinline__ void oz_cp16(void* dst, const void* src) {
    const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(d), "l"(src) : "memory");
}

// Stage tile `tile` (block rows j0 .. j0 + kOzRows - 1) into buffer st.
__device__ __forceinline__ void oz_stage(double* st, long long tile, long long N, int nr, const double* B,
                                         const double* D, const double* C, const double* X, const double* F) {
    constexpr int MM = 256;
    const long long j0 = tile * kOzRows;
    const int g = (int)((N - j0 < kOzRows) ? (N - j0) : kOzRows);
    double* sA = st;
    double* sX = st + kOzRows * 3 * kOzBlk;
    double* sF = sX + (kOzRows + 2) * 16 * nr;
    // A: block (w, kt) row r = 16 doubles = 8 chunks of 16 bytes
    for (int c = threadIdx.x; c < g * 3 * 16 * 8; c += blockDim.x) {
        const int ch = c & 7, r = (c >> 3) & 15, blk = c >> 7, w = blk / 3, kt = blk % 3;
        const double* src = (kt == 0 ? B : kt == 1 ? D : C) + (j0 + w) * MM + r * 16 + 2 * ch;
        oz_cp16(sA + (w * 3 + kt) * kOzBlk + r * kOzLd + 2 * ch, src);
    }
    // x rows j0-1 .. j0+g (those inside 0..N-1), f rows j0 .. j0+g-1: 16 nr doubles per block row
    const int v2 = 8 * nr;   // 16-byte chunks per block row
    const long long x0 = j0 - 1 < 0 ? 0 : j0 - 1, x1 = (j0 + g + 1 < N) ? j0 + g + 1 : N;
    for (int c = threadIdx.x; c < (int)(x1 - x0) * v2; c += blockDim.x) {
        const long long row = x0 + c / v2;
        oz_cp16(sX + (row - (j0 - 1)) * 16 * nr + 2 * (c % v2), X + row * 16 * nr + 2 * (c % v2));
    }
    for (int c = threadIdx.x; c < g * v2; c += blockDim.x)
        oz_cp16(sF + 2 * c, F + j0 * 16 * nr + 2 * c);
    asm volatile("cp.async.commit_group;\n" ::: "memory");
}

__global__ void __launch_bounds__(kOzThreads, 1) k_resid_btri_oz16(long long N, int nr, const double* __restrict__ B,
                                                                   const double* __restrict__ D,
                                                                   const double* __restrict__ C,
                                                                   const double* __restrict__ X,
                                                                   const double* __restrict__ F,
                                                                   double* __restrict__ R,
                                                                   unsigned long long* maxout) {
    constexpr int M = 16;
    extern __shared__ __align__(16) double oz_sm[];
    const int lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3, warp = threadIdx.x >> 5;
    const long long ntiles = (N + kOzRows - 1) / kOzRows;
    const int SD = oz_stage_doubles(nr);
    unsigned long long mr = 0ull, mx = 0ull, mf = 0ull;
    long long tile = blockIdx.x;
    if (tile < ntiles) oz_stage(oz_sm, tile, N, nr, B, D, C, X, F);
    for (int it = 0; tile < ntiles; ++it, tile += gridDim.x) {
        double* st = oz_sm + (it & 1) * SD;
        const long long nxt = tile + gridDim.x;
        if (nxt < ntiles) {
            oz_stage(oz_sm + ((it + 1) & 1) * SD, nxt, N, nr, B, D, C, X, F);
            asm volatile("cp.async.wait_group 1;\n" ::: "memory");
        } else {
            asm volatile("cp.async.wait_group 0;\n" ::: "memory");
        }
        __syncthreads();
        const long long j = tile * kOzRows + warp;
        if (j < N) {
        const double* sA = st + warp * 3 * kOzBlk;
        const double* sX = st + kOzRows * 3 * kOzBlk + warp * 16 * nr;   // window rows j-1, j, j+1
        const double* sF = st + kOzRows * 3 * kOzBlk + (kOzRows + 2) * 16 * nr + warp * 16 * nr;
        double a[3][8], xv[3][4];
#pragma unroll
        for (int kt = 0; kt < 3; ++kt) {
            const bool present = (kt == 0) ? (j > 0) : (kt == 2) ? (j + 1 < N) : true;
            const double* blk = sA + kt * kOzBlk;
            if (present) {
                const double2 u0 = *reinterpret_cast<const double2*>(blk + g * kOzLd + 2 * t);
                const double2 u1 = *reinterpret_cast<const double2*>(blk + (g + 8) * kOzLd + 2 * t);
                const double2 u2 = *reinterpret_cast<const double2*>(blk + g * kOzLd + 2 * t + 8);
                const double2 u3 = *reinterpret_cast<const double2*>(blk + (g + 8) * kOzLd + 2 * t + 8);
                a[kt][0] = u0.x; a[kt][1] = u0.y; a[kt][2] = u1.x; a[kt][3] = u1.y;
                a[kt][4] = u2.x; a[kt][5] = u2.y; a[kt][6] = u3.x; a[kt][7] = u3.y;
            } else {
#pragma unroll
                for (int e = 0; e < 8; ++e) a[kt][e] = 0.0;
            }
            const bool col = g < nr;
#pragma unroll
            for (int e = 0; e < 4; ++e) {
                const int k = 2 * t + (e & 1) + 8 * (e >> 1);
                xv[kt][e] = (present && col) ? sX[(kt * 16 + k) * nr + g] : 0.0;
            }
        }
        // scales: row maxima (rows g, g+8) and the window's column maximum (column g)
        int ea0 = 0, ea1 = 0, ex = 0;
#pragma unroll
        for (int kt = 0; kt < 3; ++kt) {
            ea0 = max(ea0, max(max(oz_expo(a[kt][0]), oz_expo(a[kt][1])), max(oz_expo(a[kt][4]), oz_expo(a[kt][5]))));
            ea1 = max(ea1, max(max(oz_expo(a[kt][2]), oz_expo(a[kt][3])), max(oz_expo(a[kt][6]), oz_expo(a[kt][7]))));
#pragma unroll
            for (int e = 0; e < 4; ++e) {
                ex = max(ex, oz_expo(xv[kt][e]));
                mx = umax_(mx, abs_bits64(xv[kt][e]));
            }
        }
#pragma unroll
        for (int o = 1; o < 4; o <<= 1) {
            ea0 = max(ea0, __shfl_xor_sync(0xffffffffu, ea0, o));
            ea1 = max(ea1, __shfl_xor_sync(0xffffffffu, ea1, o));
            ex = max(ex, __shfl_xor_sync(0xffffffffu, ex, o));
        }
        // digit-plane products, accumulated per weight t = p + q
        float acc[9][4];
#pragma unroll
        for (int u = 0; u < 9; ++u)
#pragma unroll
            for (int e = 0; e < 4; ++e) acc[u][e] = 0.f;
#pragma unroll
        for (int kt = 0; kt < 3; ++kt) {
            unsigned af[7][4], bf[7][2];
            {
                float d0[7], d1[7];
#pragma unroll
                for (int r = 0; r < 4; ++r) {
                    const int eb = (r & 1) ? ea1 : ea0;   // registers 1 and 3 hold row g + 8
                    oz_digits(a[kt][2 * r], eb, d0);
                    oz_digits(a[kt][2 * r + 1], eb, d1);
#pragma unroll
                    for (int p = 0; p < 7; ++p) af[p][r] = oz_pack(d0[p], d1[p]);
                }
#pragma unroll
                for (int r = 0; r < 2; ++r) {
                    oz_digits(xv[kt][2 * r], ex, d0);
                    oz_digits(xv[kt][2 * r + 1], ex, d1);
#pragma unroll
                    for (int q = 0; q < 7; ++q) bf[q][r] = oz_pack(d0[q], d1[q]);
                }
            }
#pragma unroll
            for (int p = 0; p < 7; ++p)
#pragma unroll
                for (int q = 0; q < 7; ++q) {
                    if (p + q > 7) continue;
                    const int w = p + q;
                    // accumulator of weight w (weight 5 split in two: at most 3 plane pairs each)
                    const int slot = (w < 5) ? w : (w == 5) ? (p < 3 ? 5 : 6) : w + 1;
                    oz_mma(acc[slot], af[p], bf[q][0], bf[q][1]);
                }
        }
        // r = f - (sum_w acc_w 2^(56 - 8w)) 2^(E_row + F_col - 70), in double-float
        const float wts[9] = {0x1p56f, 0x1p48f, 0x1p40f, 0x1p32f, 0x1p24f, 0x1p16f, 0x1p16f, 0x1p8f, 1.f};
        // the other lanes' column exponents: outputs of this lane are columns 2t, 2t+1
        const int exc0 = __shfl_sync(0xffffffffu, ex, 4 * (2 * t));
        const int exc1 = __shfl_sync(0xffffffffu, ex, 4 * (2 * t + 1));
#pragma unroll
        for (int e = 0; e < 4; ++e) {
            const int row = (e < 2) ? g : g + 8;
            const int colw = 2 * t + (e & 1);
            if (colw >= nr) continue;
            float sh = 0.f, sl = 0.f;
#pragma unroll
            for (int u = 8; u >= 0; --u) {
                float err;
                two_sum(sh, acc[u][e] * wts[u], sh, err);
                sl = __fadd_rn(sl, err);
            }
            const int eb = ((e < 2) ? ea0 : ea1) + ((e & 1) ? exc1 : exc0) - 2046;   // E_row + F_col (unbiased sum)
            const long long orow = j * M + row;
            const double fv = sF[row * nr + colw];
            mf = umax_(mf, abs_bits64(fv));
            const int k = eb - 70;
            double rv;
            if (k > -100 && k < 40) {
                const float sc = __uint_as_float((unsigned)(k + 127) << 23);
                const float2 fs = split_f64(fv);
                float u, ue;
                two_sum(fs.x, -(sh * sc), u, ue);
                const float low = __fadd_rn(__fsub_rn(fs.y, sl * sc), ue);
                rv = f32_to_f64(__fadd_rn(u, low));
            } else {
                // far outside the FP32 range of the scaled sum: FP64 arithmetic
                rv = fv - ldexp(f32_to_f64(sh) + f32_to_f64(sl), k);
            }
            if (oz_expo(fv) == 0x7ff || ((e < 2) ? ea0 : ea1) == 0x7ff || ((e & 1) ? exc1 : exc0) == 0x7ff)
                rv = fv + __longlong_as_double(0x7ff8000000000000ll);   // non-finite operands
            R[orow * nr + colw] = rv;
            mr = umax_(mr, abs_bits64(rv));
        }
        }
        __syncthreads();   // the buffer is refilled by the next iteration's staging
    }
    if (maxout) block_max3_df(mr, mx, mf, maxout);
}

}  // namespace

static size_t resid_dfs_smem(int m, int nr, int G) {
    const int pcp = 1 << df_pair_shift(nr), V = m * nr;
    const size_t nA = (size_t)G * 3 * m * m, nX = (size_t)(G + 2) * V, nF = (size_t)G * V;
    return 2 * nA * sizeof(float2) + 2 * (nX + nF) * sizeof(double) + (size_t)(G + 2) * m * pcp * sizeof(float4);
}

cudaError_t launch_resid_btri_oz(long long N, int m, int nr, const double* B, const double* D, const double* C,
                                 const double* X, const double* F, double* R, cudaStream_t s,
                                 unsigned long long* maxout) {
    if (N <= 0) return cudaSuccess;
    if (m != 16 || nr < 1 || nr > 8 || (((uintptr_t)B | (uintptr_t)D | (uintptr_t)C) & 15u)) return cudaErrorInvalidValue;
    int dev = 0, sms = 148;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (((uintptr_t)X | (uintptr_t)F) & 15u) return cudaErrorInvalidValue;
    const long long ntiles = (N + kOzRows - 1) / kOzRows;
    long long grid = ntiles < sms ? ntiles : sms;
    const size_t smem = 2 * sizeof(double) * (size_t)oz_stage_doubles(nr);
    cudaError_t e = cudaFuncSetAttribute(k_resid_btri_oz16, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    k_resid_btri_oz16<<<(unsigned)grid, kOzThreads, smem, s>>>(N, nr, B, D, C, X, F, R, maxout);
    return cudaGetLastError();
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
