// FP64 residuals, the refinement update with deterministic norms, and the
// direct solver for the small BABD system at the top of the recursion.
#include <cuda_runtime.h>
#include "../../include/bt.h"
#include "bt_device.cuh"
#include "bt_misc.h"

namespace bt {

// |v| as an integer key: the bit pattern with the sign cleared orders
// non-negative doubles like their values (integer pipes only, no FP64 work).
__device__ __forceinline__ unsigned long long abs_bits(double v) {
    return (unsigned long long)__double_as_longlong(v) & 0x7fffffffffffffffull;
}
__device__ __forceinline__ unsigned long long umax64(unsigned long long a, unsigned long long b) {
    return a > b ? a : b;
}

// Largest of the keys r, x, f over the block, merged into slot (block mod
// kMaxSlots) of out with an integer atomicMax (order-independent).  Every
// thread of the block must call it, from one call site.
__device__ __forceinline__ void block_max3(unsigned long long r, unsigned long long x, unsigned long long f,
                                           unsigned long long* out) {
    __shared__ unsigned long long sm[3][8];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
        r = umax64(r, __shfl_xor_sync(0xffffffffu, r, off));
        x = umax64(x, __shfl_xor_sync(0xffffffffu, x, off));
        f = umax64(f, __shfl_xor_sync(0xffffffffu, f, off));
    }
    if (lane == 0) {
        sm[0][warp] = r;
        sm[1][warp] = x;
        sm[2][warp] = f;
    }
    __syncthreads();
    if (threadIdx.x < 3) {
        unsigned long long v = 0ull;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) v = umax64(v, sm[threadIdx.x][w]);
        atomicMax(out + 3 * (blockIdx.x % kMaxSlots) + threadIdx.x, v);
    }
}

// r = f - A x for the block tridiagonal A; one thread per entry of [N*m][nr].
__global__ void __launch_bounds__(256) k_resid_btri(long long N, int m, int nr, const double* __restrict__ B,
                                                    const double* __restrict__ D, const double* __restrict__ C,
                                                    const double* __restrict__ X, const double* __restrict__ F,
                                                    double* __restrict__ R, unsigned long long* maxout) {
    const long long el = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const long long total = N * m * nr;
    unsigned long long ar = 0ull, ax = 0ull, af = 0ull;
    if (el < total) {
        const long long gr = el / nr;
        const int c = (int)(el % nr);
        const long long j = gr / m;
        const int r = (int)(gr % m);
        const long long mm = (long long)m * m;
        double acc = F[el];
        const double* Drow = D + j * mm + (long long)r * m;
        const double* xj = X + j * m * nr + c;
        for (int k = 0; k < m; ++k) acc = fma(-Drow[k], xj[(long long)k * nr], acc);
        if (j > 0) {
            const double* Brow = B + j * mm + (long long)r * m;
            const double* xp = xj - (long long)m * nr;
            for (int k = 0; k < m; ++k) acc = fma(-Brow[k], xp[(long long)k * nr], acc);
        }
        if (j + 1 < N) {
            const double* Crow = C + j * mm + (long long)r * m;
            const double* xn = xj + (long long)m * nr;
            for (int k = 0; k < m; ++k) acc = fma(-Crow[k], xn[(long long)k * nr], acc);
        }
        R[el] = acc;
        ar = abs_bits(acc);
        ax = abs_bits(X[el]);
        af = abs_bits(F[el]);
    }
    // every thread of the block reaches this one call site (warp shuffles and
    // the block barrier inside must not be split across branches)
    if (maxout) block_max3(ar, ax, af, maxout);
}

// r = f - A y for the BABD A (rows 0..N, boundary row first).
__global__ void __launch_bounds__(256) k_resid_babd(long long N, int m, int nr, const double* __restrict__ S,
                                                    const double* __restrict__ Rm, const double* __restrict__ B0,
                                                    const double* __restrict__ B1, const double* __restrict__ Y,
                                                    const double* __restrict__ F, double* __restrict__ Rout,
                                                    unsigned long long* maxout) {
    const long long el = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const long long total = (N + 1) * m * nr;
    unsigned long long ar = 0ull, ay = 0ull, af = 0ull;
    if (el < total) {
        const long long gr = el / nr;
        const int c = (int)(el % nr);
        const long long j = gr / m;
        const int r = (int)(gr % m);
        const long long mm = (long long)m * m;
        double acc = F[el];
        if (j == 0) {
            const double* y0 = Y + c;
            const double* yN = Y + N * m * nr + c;
            for (int k = 0; k < m; ++k) {
                acc = fma(-B0[r * m + k], y0[(long long)k * nr], acc);
                acc = fma(-B1[r * m + k], yN[(long long)k * nr], acc);
            }
        } else {
            const double* Srow = S + (j - 1) * mm + (long long)r * m;
            const double* Rrow = Rm + (j - 1) * mm + (long long)r * m;
            const double* yp = Y + (j - 1) * m * nr + c;
            const double* yj = Y + j * m * nr + c;
            for (int k = 0; k < m; ++k) {
                acc = fma(-Srow[k], yp[(long long)k * nr], acc);
                acc = fma(-Rrow[k], yj[(long long)k * nr], acc);
            }
        }
        Rout[el] = acc;
        ar = abs_bits(acc);
        ay = abs_bits(Y[el]);
        af = abs_bits(F[el]);
    }
    if (maxout) block_max3(ar, ay, af, maxout);   // one call site for the whole block
}

// |v| truncated to FP32 by integer operations (no FP64 work): exponent
// rebiased, mantissa cut to its top 20 bits, magnitudes below the FP32 normal
// range flushed to zero and above it clamped to 2^127.  Never above |v|.
__device__ __forceinline__ float abs_trunc_f32(double v) {
    const unsigned hi = (unsigned)__double2hiint(v) & 0x7fffffffu;
    const int e = (int)(hi >> 20) - 1023 + 127;
    if (e <= 0) return 0.0f;
    if (e >= 255) return __uint_as_float(254u << 23);
    return __uint_as_float(((unsigned)e << 23) | ((hi & 0xfffffu) << 3));
}

// ||A||_inf = max row sum of |A| (block tridiagonal: B, D, C rows; BABD:
// row block 0 = [B0 | B1], row block j+1 = [S_j | R_j]), in FP32 from entries
// truncated toward zero: relative error below 1e-5 (it only enters the
// backward-error stopping threshold, where a slightly smaller norm makes the
// test slightly stricter).  The
// blocks are row-major, so each array is a list of rows of m contiguous
// entries; lane l of a warp takes entry 32w + l, a warp step covers 32/m whole
// rows (m divides 32) with coalesced loads, and a shuffle reduction over each
// group of m lanes finishes the row sums.
__global__ void __launch_bounds__(256) k_norm_inf(int kind, long long N, int m, const double* __restrict__ A0,
                                                  const double* __restrict__ A1, const double* __restrict__ A2,
                                                  const double* __restrict__ B0, const double* __restrict__ B1,
                                                  unsigned long long* out) {
    const long long rows = (kind == 0) ? N * m : (N + 1) * m;
    const long long total = rows * m;
    const long long mm = (long long)m * m;
    const int lane = threadIdx.x & 31;
    const long long warps = (long long)gridDim.x * (blockDim.x >> 5);
    float best = 0.0f;
    for (long long base = ((long long)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5)) * 32; base < total;
         base += warps * 32) {   // uniform within the warp
        const long long e = base + lane;
        float s = 0.0f;
        if (e < total) {
            const long long j = e / mm;
            if (kind == 0) {
                s = abs_trunc_f32(A1[e]);
                if (j > 0) s += abs_trunc_f32(A0[e]);
                if (j + 1 < N) s += abs_trunc_f32(A2[e]);
            } else if (j == 0) {
                s = abs_trunc_f32(B0[e]) + abs_trunc_f32(B1[e]);
            } else {
                s = abs_trunc_f32(A0[e - mm]) + abs_trunc_f32(A1[e - mm]);
            }
        }
        for (int off = 1; off < m; off <<= 1) s += __shfl_xor_sync(0xffffffffu, s, off);
        best = fmaxf(best, s);
    }
    // as a double bit pattern so that the slots hold doubles like the residual maxima
    block_max3(abs_bits((double)best), 0ull, 0ull, out);
}

// x += d; per-block partial sums of |d|^2 and |x|^2 (after the update).
__global__ void __launch_bounds__(256) k_ir_update(long long n, double* __restrict__ X,
                                                   const double* __restrict__ Dc, double* __restrict__ partial) {
    __shared__ double sd[256], sx[256];
    double ad = 0.0, ax = 0.0;
    for (long long el = (long long)blockIdx.x * blockDim.x + threadIdx.x; el < n;
         el += (long long)gridDim.x * blockDim.x) {
        const double d = Dc[el];
        const double x = X[el] + d;
        X[el] = x;
        ad = fma(d, d, ad);
        ax = fma(x, x, ax);
    }
    sd[threadIdx.x] = ad;
    sx[threadIdx.x] = ax;
    __syncthreads();
    for (int s = 128; s > 0; s >>= 1) {
        if (threadIdx.x < s) {
            sd[threadIdx.x] += sd[threadIdx.x + s];
            sx[threadIdx.x] += sx[threadIdx.x + s];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        partial[2 * blockIdx.x] = sd[0];
        partial[2 * blockIdx.x + 1] = sx[0];
    }
}

__global__ void __launch_bounds__(256) k_reduce_pairs(int nblocks, const double* __restrict__ partial,
                                                      double* __restrict__ out) {
    __shared__ double sd[256], sx[256];
    double ad = 0.0, ax = 0.0;
    for (int b = threadIdx.x; b < nblocks; b += blockDim.x) {
        ad += partial[2 * b];
        ax += partial[2 * b + 1];
    }
    sd[threadIdx.x] = ad;
    sx[threadIdx.x] = ax;
    __syncthreads();
    for (int s = 128; s > 0; s >>= 1) {
        if (threadIdx.x < s) {
            sd[threadIdx.x] += sd[threadIdx.x + s];
            sx[threadIdx.x] += sx[threadIdx.x + s];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        out[0] = sd[0];
        out[1] = sx[0];
    }
}

// Direct solve of a small BABD system (rows 0..Np: B0 y_0 + B1 y_Np = f_0;
// S_j y_j + R_j y_{j+1} = f_{j+1}) in one CTA by Gaussian elimination with
// partial pivoting restricted to the rows that are nonzero in each pivot
// column: m rows carried from the previous step (initially the boundary
// rows, which carry the corner fill-in) and the m rows of block row j+1.
// Columns of the working rows: [y_j | y_{j+1} | y_Np | rhs].
// keep: workspace of Np * m * (3m + nr) doubles for the pivot rows.
__global__ void __launch_bounds__(256) k_babd_direct(int Np, int m, int nr, const double* __restrict__ S,
                                                     const double* __restrict__ R, const double* __restrict__ B0,
                                                     const double* __restrict__ B1, const double* __restrict__ F,
                                                     double* __restrict__ X, double* __restrict__ keep,
                                                     long long* status, int level) {
    extern __shared__ __align__(16) double sm[];
    const int W = 3 * m + nr, H = 2 * m;
    double* w = sm;
    double* colk = w + H * W;
    const int tid = threadIdx.x, NT = blockDim.x, lane = tid & 31, warp = tid >> 5;
    const long long mm = (long long)m * m;
    const int MW = m * W;
    for (int idx = tid; idx < MW; idx += NT) {
        const int r = idx / W, c = idx % W;
        double v;
        if (c < m) v = B0[r * m + c];
        else if (c < 2 * m) v = 0.0;
        else if (c < 3 * m) v = B1[r * m + (c - 2 * m)];
        else v = F[r * nr + (c - 3 * m)];
        w[idx] = v;
    }
    __syncthreads();
    for (int j = 0; j < Np; ++j) {
        const bool last = (j + 1 == Np);
        for (int idx = tid; idx < MW; idx += NT) {
            const int r = idx / W, c = idx % W;
            double v;
            if (c < m) v = S[j * mm + r * m + c];
            else if (c < 2 * m) v = last ? 0.0 : R[j * mm + r * m + (c - m)];
            else if (c < 3 * m) v = last ? R[j * mm + r * m + (c - 2 * m)] : 0.0;
            else v = F[((long long)(j + 1) * m + r) * nr + (c - 3 * m)];
            w[MW + idx] = v;
        }
        __syncthreads();
        for (int k = 0; k < m; ++k) {
            if (warp == 0) {
                unsigned long long key = 0ull;
                int idx = 1 << 20;
                for (int i = lane; i < H; i += 32) {
                    if (i >= k) {
                        const unsigned long long kk = abs_key(w[i * W + k]);
                        if (kk > key || (kk == key && i < idx)) {
                            key = kk;
                            idx = i;
                        }
                    }
                }
#pragma unroll
                for (int off = 16; off > 0; off >>= 1) {
                    const unsigned long long k2 = __shfl_xor_sync(0xffffffffu, key, off);
                    const int i2 = __shfl_xor_sync(0xffffffffu, idx, off);
                    if (k2 > key || (k2 == key && i2 < idx)) {
                        key = k2;
                        idx = i2;
                    }
                }
                const int p = idx;
                if (p != k)
                    for (int c = lane; c < W; c += 32) {
                        const double t = w[k * W + c];
                        w[k * W + c] = w[p * W + c];
                        w[p * W + c] = t;
                    }
                __syncwarp();
                double pv = w[k * W + k];
                if (key == 0ull || nonfinite(pv)) {
                    if (lane == 0) report(status, key == 0ull ? ST_SINGULAR : ST_NONFINITE, level, -1, j);
                    pv = 1.0;
                }
                const double rp = rcp(pv);
                for (int i = lane; i < H; i += 32) colk[i] = (i > k) ? w[i * W + k] * rp : 0.0;
            }
            __syncthreads();
            const int rows = H - k - 1, cols = W - k - 1;
            for (int idx = tid; idx < rows * cols; idx += NT) {
                const int i = k + 1 + idx / cols, c = k + 1 + idx % cols;
                w[i * W + c] = fma(-colk[i], w[k * W + c], w[i * W + c]);
            }
            for (int i = k + 1 + tid; i < H; i += NT) w[i * W + k] = 0.0;
            __syncthreads();
        }
        double* kp = keep + (long long)j * MW;
        for (int idx = tid; idx < MW; idx += NT) kp[idx] = w[idx];
        __syncthreads();
        double tmp[16];
        int u = 0;
        for (int idx = tid; idx < MW; idx += NT, ++u) {
            const int r = idx / W, c = idx % W;
            const double* src = w + (m + r) * W;
            double v;
            if (c < m) v = src[m + c];
            else if (c < 2 * m) v = 0.0;
            else v = src[c];
            tmp[u] = v;
        }
        __syncthreads();
        u = 0;
        for (int idx = tid; idx < MW; idx += NT, ++u) w[idx] = tmp[u];
        __syncthreads();
    }
    // final m x m system in y_Np: Gauss-Jordan with partial pivoting on rows 0..m-1
    for (int k = 0; k < m; ++k) {
        const int ck = 2 * m + k;
        if (warp == 0) {
            unsigned long long key = 0ull;
            int idx = 1 << 20;
            if (lane >= k && lane < m) {
                key = abs_key(w[lane * W + ck]);
                idx = lane;
            }
#pragma unroll
            for (int off = 16; off > 0; off >>= 1) {
                const unsigned long long k2 = __shfl_xor_sync(0xffffffffu, key, off);
                const int i2 = __shfl_xor_sync(0xffffffffu, idx, off);
                if (k2 > key || (k2 == key && i2 < idx)) {
                    key = k2;
                    idx = i2;
                }
            }
            const int p = idx;
            if (p != k)
                for (int c = lane; c < W; c += 32) {
                    const double t = w[k * W + c];
                    w[k * W + c] = w[p * W + c];
                    w[p * W + c] = t;
                }
            __syncwarp();
            double pv = w[k * W + ck];
            if (key == 0ull || nonfinite(pv)) {
                if (lane == 0) report(status, key == 0ull ? ST_SINGULAR : ST_NONFINITE, level, -1, Np);
                pv = 1.0;
            }
            const double rp = rcp(pv);
            __syncwarp();
            for (int c = 2 * m + lane; c < W; c += 32) w[k * W + c] = (c == ck) ? 1.0 : w[k * W + c] * rp;
            __syncwarp();
            for (int i = lane; i < m; i += 32) colk[i] = (i == k) ? 0.0 : w[i * W + ck];
        }
        __syncthreads();
        const int cols = W - 2 * m;
        for (int idx = tid; idx < m * cols; idx += NT) {
            const int i = idx / cols, c = 2 * m + idx % cols;
            if (i != k) w[i * W + c] = fma(-colk[i], w[k * W + c], w[i * W + c]);
        }
        __syncthreads();
    }
    const long long E = (long long)m * nr;
    for (int idx = tid; idx < m * nr; idx += NT) {
        const int r = idx / nr, c = idx % nr;
        X[(long long)Np * E + idx] = w[r * W + 3 * m + c];
    }
    __syncthreads();
    // back substitution: U_j y_j = rhs_j - P_j y_{j+1} - Q_j y_Np
    double* t = w;   // m x nr
    for (int j = Np - 1; j >= 0; --j) {
        const double* kp = keep + (long long)j * MW;
        const double* y1 = X + (long long)(j + 1) * E;
        const double* yN = X + (long long)Np * E;
        const bool last = (j + 1 == Np);
        for (int idx = tid; idx < m * nr; idx += NT) {
            const int r = idx / nr, c = idx % nr;
            double acc = kp[r * W + 3 * m + c];
            for (int k = 0; k < m; ++k) {
                if (!last) acc = fma(-kp[r * W + m + k], y1[k * nr + c], acc);
                acc = fma(-kp[r * W + 2 * m + k], yN[k * nr + c], acc);
            }
            t[idx] = acc;
        }
        __syncthreads();
        double* yj = X + (long long)j * E;
        for (int c = tid; c < nr; c += NT) {
            for (int r = m - 1; r >= 0; --r) {
                double acc = t[r * nr + c];
                for (int k = r + 1; k < m; ++k) acc = fma(-kp[r * W + k], t[k * nr + c], acc);
                acc = acc * rcp(kp[r * W + r]);
                t[r * nr + c] = acc;
                yj[r * nr + c] = acc;
            }
        }
        __syncthreads();
    }
}

// Direct solve of a small block tridiagonal system (K block rows) by Gaussian
// elimination with partial pivoting, row interchanges being confined to two
// consecutive block rows (the banded form of GEPP: after the interchanges, row
// block j of U reaches block columns j, j+1 and j+2).  One CTA.  The working
// window holds 2m rows of [x_j | x_{j+1} | x_{j+2} | f]; per block column the
// m pivot rows go to keep ([K][m][3m+nr]) for the back substitution.  The
// top of a pivoted recursion, where a reduced system may have singular
// diagonal blocks that block elimination without interchanges cannot pass.
__global__ void __launch_bounds__(256) k_btri_direct(int K, int m, int nr, const double* __restrict__ B,
                                                     const double* __restrict__ D, const double* __restrict__ C,
                                                     const double* __restrict__ F, double* __restrict__ X,
                                                     double* __restrict__ keep, long long* status, int level) {
    extern __shared__ __align__(16) double sm[];
    const int W = 3 * m + nr;
    double* w = sm;
    double* colk = w + 2 * m * W;
    const int tid = threadIdx.x, NT = blockDim.x, lane = tid & 31, warp = tid >> 5;
    const long long mm = (long long)m * m;
    const int MW = m * W;
    // block row j in the window frame of block column j-1 (rows m..2m-1) or j (rows 0..m-1)
    auto load_row = [&](int j, double* dst, bool shifted) {
        for (int idx = tid; idx < MW; idx += NT) {
            const int r = idx / W, c = idx % W;
            double v = 0.0;
            if (c < 3 * m) {
                const int blk = c / m, cc = c % m;   // window block column
                const int col = shifted ? (j - 1 + blk) : (j + blk);
                if (col == j - 1) v = B[j * mm + r * m + cc];
                else if (col == j) v = D[j * mm + r * m + cc];
                else if (col == j + 1 && j + 1 < K) v = C[j * mm + r * m + cc];
            } else {
                v = F[((long long)j * m + r) * nr + (c - 3 * m)];
            }
            dst[idx] = v;
        }
    };
    load_row(0, w, false);
    __syncthreads();
    for (int j = 0; j < K; ++j) {
        const bool more = (j + 1 < K);
        if (more) load_row(j + 1, w + MW, true);
        __syncthreads();
        const int H = more ? 2 * m : m;
        for (int k = 0; k < m; ++k) {
            if (warp == 0) {
                unsigned long long key = 0ull;
                int idx = 1 << 20;
                for (int i = k + lane; i < H; i += 32) {
                    const unsigned long long kk = abs_key(w[i * W + k]);
                    if (kk > key || (kk == key && i < idx)) {
                        key = kk;
                        idx = i;
                    }
                }
#pragma unroll
                for (int off = 16; off > 0; off >>= 1) {
                    const unsigned long long k2 = __shfl_xor_sync(0xffffffffu, key, off);
                    const int i2 = __shfl_xor_sync(0xffffffffu, idx, off);
                    if (k2 > key || (k2 == key && i2 < idx)) {
                        key = k2;
                        idx = i2;
                    }
                }
                const int p = (idx < H) ? idx : k;
                if (p != k)
                    for (int c = lane; c < W; c += 32) {
                        const double t = w[k * W + c];
                        w[k * W + c] = w[p * W + c];
                        w[p * W + c] = t;
                    }
                __syncwarp();
                double pv = w[k * W + k];
                if (key == 0ull || nonfinite(pv)) {
                    if (lane == 0) report(status, key == 0ull ? ST_SINGULAR : ST_NONFINITE, level, -1, j);
                    pv = 1.0;
                    if (lane == 0) w[k * W + k] = 1.0;
                }
                const double rp = rcp(pv);
                for (int i = lane; i < H; i += 32) colk[i] = (i > k) ? w[i * W + k] * rp : 0.0;
            }
            __syncthreads();
            const int rows = H - k - 1, cols = W - k - 1;
            for (int idx = tid; idx < rows * cols; idx += NT) {
                const int i = k + 1 + idx / cols, c = k + 1 + idx % cols;
                w[i * W + c] = fma(-colk[i], w[k * W + c], w[i * W + c]);
            }
            for (int i = k + 1 + tid; i < H; i += NT) w[i * W + k] = 0.0;
            __syncthreads();
        }
        double* kp = keep + (long long)j * MW;
        for (int idx = tid; idx < MW; idx += NT) kp[idx] = w[idx];
        __syncthreads();
        if (more) {
            // the m rows left over move up one block column: [x_{j+1} | x_{j+2} | 0 | f]
            for (int idx = tid; idx < MW; idx += NT) {
                const int r = idx / W, c = idx % W;
                const double* src = w + (m + r) * W;
                double v;
                if (c < 2 * m) v = src[m + c];
                else if (c < 3 * m) v = 0.0;
                else v = src[c];
                w[idx] = v;   // rows 0..m-1 are not read again in this pass
            }
            __syncthreads();
        }
    }
    // back substitution: x_j = U_jj^{-1} (g_j - U_{j,j+1} x_{j+1} - U_{j,j+2} x_{j+2}), U_jj upper triangular
    const long long E = (long long)m * nr;
    double* t = w;   // m x nr
    for (int j = K - 1; j >= 0; --j) {
        const double* kp = keep + (long long)j * MW;
        for (int el = tid; el < m * nr; el += NT) {
            const int r = el / nr, c = el % nr;
            double acc = kp[r * W + 3 * m + c];
            if (j + 1 < K)
                for (int k = 0; k < m; ++k) acc = fma(-kp[r * W + m + k], X[(long long)(j + 1) * E + k * nr + c], acc);
            if (j + 2 < K)
                for (int k = 0; k < m; ++k)
                    acc = fma(-kp[r * W + 2 * m + k], X[(long long)(j + 2) * E + k * nr + c], acc);
            t[el] = acc;
        }
        __syncthreads();
        for (int r = m - 1; r >= 0; --r) {
            for (int c = tid; c < nr; c += NT) {
                double acc = t[r * nr + c];
                for (int k = r + 1; k < m; ++k) acc = fma(-kp[r * W + k], t[k * nr + c], acc);
                t[r * nr + c] = acc * rcp(kp[r * W + r]);
            }
            __syncthreads();
        }
        for (int el = tid; el < m * nr; el += NT) X[(long long)j * E + el] = t[el];
        __syncthreads();
    }
}

size_t babd_direct_smem(int m, int nr) { return sizeof(double) * ((size_t)(2 * m) * (3 * m + nr) + 2 * m); }

cudaError_t launch_resid_btri(long long N, int m, int nr, const double* B, const double* D, const double* C,
                              const double* X, const double* F, double* R, cudaStream_t s,
                              unsigned long long* maxout) {
    const long long total = N * m * nr;
    if (total == 0) return cudaSuccess;
    k_resid_btri<<<(unsigned)((total + 255) / 256), 256, 0, s>>>(N, m, nr, B, D, C, X, F, R, maxout);
    return cudaGetLastError();
}
cudaError_t launch_resid_babd(long long N, int m, int nr, const double* S, const double* Rm, const double* B0,
                              const double* B1, const double* Y, const double* F, double* Rout, cudaStream_t s,
                              unsigned long long* maxout) {
    const long long total = (N + 1) * m * nr;
    k_resid_babd<<<(unsigned)((total + 255) / 256), 256, 0, s>>>(N, m, nr, S, Rm, B0, B1, Y, F, Rout, maxout);
    return cudaGetLastError();
}
cudaError_t launch_norm_inf(int kind, long long N, int m, const double* A0, const double* A1, const double* A2,
                            const double* B0, const double* B1, unsigned long long* out, cudaStream_t s) {
    if (m < 1 || m > 32 || (32 % m) != 0) return cudaErrorInvalidValue;
    const long long total = ((kind == 0) ? N * m : (N + 1) * m) * m;
    long long nb = (total + 255) / 256;
    if (nb > 2048) nb = 2048;
    if (nb < 1) nb = 1;
    k_norm_inf<<<(unsigned)nb, 256, 0, s>>>(kind, N, m, A0, A1, A2, B0, B1, out);
    return cudaGetLastError();
}
int ir_update_blocks(long long n) {
    long long b = (n + 255) / 256;
    if (b > 1024) b = 1024;
    if (b < 1) b = 1;
    return (int)b;
}
cudaError_t launch_reduce_pairs(int n, const double* partial, double* out, cudaStream_t s) {
    k_reduce_pairs<<<1, 256, 0, s>>>(n, partial, out);
    return cudaGetLastError();
}

cudaError_t launch_ir_update(long long n, double* X, const double* Dc, double* partial, double* out,
                             cudaStream_t s) {
    const int nb = ir_update_blocks(n);
    k_ir_update<<<nb, 256, 0, s>>>(n, X, Dc, partial);
    k_reduce_pairs<<<1, 256, 0, s>>>(nb, partial, out);
    return cudaGetLastError();
}
// Scalar case (m = 1) of k_btri_direct: Gaussian elimination with partial
// pivoting on a tridiagonal matrix (row interchanges between consecutive rows
// fill in a second superdiagonal), one warp, lane c carrying right-hand side
// c; every lane takes the same pivot decisions.  keep: [K][3] rows of U
// (reciprocal of the diagonal, first and second superdiagonal), then [K][nr]
// eliminated right-hand sides.
//
// The elimination is a chain of dependent FP64 operations (a reciprocal, a
// multiplier and one update per row), so the loads are taken off it: the rows
// are fetched 32 at a time one chunk ahead into registers (lane l: row
// base + l of the matrix; every lane its own right-hand-side column of the 32
// rows), parked in shared memory while the chain walks the current chunk from
// there; the back substitution prefetches U and the eliminated right-hand
// sides the same way, downwards.
namespace {
constexpr int kGtsvChunk = 32;
struct GtsvRegs {
    double a, b, c;                 // lane l: B, D, C of row base + l (C = 0 past the last coupling)
    double f[kGtsvChunk];           // this lane's right-hand-side column of rows base .. base + 31
};
struct GtsvSmem {
    double a[kGtsvChunk], b[kGtsvChunk], c[kGtsvChunk];
    double f[kGtsvChunk][kGtsvChunk + 1];   // [row][column], padded
};
__device__ __forceinline__ void gtsv_fetch(GtsvRegs& q, long long base, long long K, int nr, bool act, int lane,
                                           const double* __restrict__ B, const double* __restrict__ D,
                                           const double* __restrict__ C, const double* __restrict__ F) {
    const long long r = base + lane;
    q.a = (r < K) ? B[r] : 0.0;
    q.b = (r < K) ? D[r] : 0.0;
    q.c = (r + 1 < K) ? C[r] : 0.0;
#pragma unroll
    for (int u = 0; u < kGtsvChunk; ++u) q.f[u] = (act && base + u < K) ? F[(base + u) * nr + lane] : 0.0;
}
__device__ __forceinline__ void gtsv_park(GtsvSmem& sm, const GtsvRegs& q, int lane) {
    sm.a[lane] = q.a;
    sm.b[lane] = q.b;
    sm.c[lane] = q.c;
#pragma unroll
    for (int u = 0; u < kGtsvChunk; ++u) sm.f[u][lane] = q.f[u];
}
// back substitution: lane l holds row top - l of U; every lane its eliminated
// right-hand-side column of rows top .. top - 31
__device__ __forceinline__ void gtsv_fetch_back(GtsvRegs& q, long long top, int nr, bool act, int lane,
                                                const double* U, const double* G) {
    const long long r = top - lane;
    q.a = (r >= 0) ? U[3 * r] : 0.0;
    q.b = (r >= 0) ? U[3 * r + 1] : 0.0;
    q.c = (r >= 0) ? U[3 * r + 2] : 0.0;
#pragma unroll
    for (int u = 0; u < kGtsvChunk; ++u) q.f[u] = (act && top - u >= 0) ? G[(top - u) * nr + lane] : 0.0;
}
}  // namespace

__global__ void __launch_bounds__(32) k_gtsv(int K, int nr, const double* __restrict__ B,
                                             const double* __restrict__ D, const double* __restrict__ C,
                                             const double* __restrict__ F, double* __restrict__ X,
                                             double* __restrict__ keep, long long* status, int level) {
    __shared__ GtsvSmem sm[2];
    const int c = threadIdx.x;
    const bool act = c < nr;
    double* U = keep;                      // [K][3]
    double* G = keep + 3 * (long long)K;   // [K][nr] eliminated right-hand sides
    // working row i: [b (diagonal), cc (super), dd (second super)] and its right-hand side
    double b = D[0], cc = (K > 1) ? C[0] : 0.0, f = act ? F[c] : 0.0;
    // chunk t holds rows i + 1 for i in [32 t, 32 t + 32)
    GtsvRegs q;
    gtsv_fetch(q, 1, K, nr, act, c, B, D, C, F);
    gtsv_park(sm[0], q, c);
    __syncwarp();
    int cb = 0;
    for (long long i0 = 0; i0 < K; i0 += kGtsvChunk) {
        gtsv_fetch(q, i0 + 1 + kGtsvChunk, K, nr, act, c, B, D, C, F);   // in flight during the chain
        const GtsvSmem& cur = sm[cb];
        const int n = (int)((K - i0 < kGtsvChunk) ? (K - i0) : kGtsvChunk);
#pragma unroll 1
        for (int u = 0; u < n; ++u) {
            const long long i = i0 + u;
            const double a1 = cur.a[u], b1 = cur.b[u], c1 = cur.c[u], f1 = cur.f[u][c];
            // magnitudes compared as integer keys: the FP64 pipe stays free for the chain
            const unsigned long long kb = abs_key(b);
            if (i + 1 < K) {
                if (kb >= abs_key(a1)) {
                    // pivot on row i: eliminate a1 from row i+1
                    double pv = b;
                    if (kb == 0ull || nonfinite(pv)) {
                        if (c == 0) report(status, kb == 0ull ? ST_SINGULAR : ST_NONFINITE, level, -1, i);
                        pv = 1.0;
                    }
                    const double rv = rcp(pv);
                    const double l = a1 * rv;
                    if (c == 0) {
                        U[3 * i] = rv;
                        U[3 * i + 1] = cc;
                        U[3 * i + 2] = 0.0;
                    }
                    if (act) G[i * nr + c] = f;
                    b = fma(-l, cc, b1);
                    cc = c1;
                    f = fma(-l, f, f1);
                } else {
                    // interchange rows i and i+1, then eliminate
                    const double rv = rcp(a1);
                    const double l = b * rv;
                    if (c == 0) {
                        U[3 * i] = rv;
                        U[3 * i + 1] = b1;
                        U[3 * i + 2] = c1;
                    }
                    if (act) G[i * nr + c] = f1;
                    const double nb = fma(-l, b1, cc);
                    cc = -l * c1;
                    b = nb;
                    f = fma(-l, f1, f);
                }
            } else {
                double pv = b;
                if (kb == 0ull || nonfinite(pv)) {
                    if (c == 0) report(status, kb == 0ull ? ST_SINGULAR : ST_NONFINITE, level, -1, i);
                    pv = 1.0;
                }
                if (c == 0) {
                    U[3 * i] = rcp(pv);
                    U[3 * i + 1] = 0.0;
                    U[3 * i + 2] = 0.0;
                }
                if (act) G[i * nr + c] = f;
            }
        }
        cb ^= 1;
        gtsv_park(sm[cb], q, c);
        __syncwarp();
    }
    // U and G come back from global memory: make this warp's stores visible to all its lanes
    __threadfence_block();
    __syncwarp();
    // back substitution: x_i = (g_i - u1_i x_{i+1} - u2_i x_{i+2}) / u0_i  (U holds 1 / u0_i)
    double x1 = 0.0, x2 = 0.0;
    gtsv_fetch_back(q, K - 1, nr, act, c, U, G);
    gtsv_park(sm[0], q, c);
    __syncwarp();
    cb = 0;
    for (long long top = K - 1; top >= 0; top -= kGtsvChunk) {
        gtsv_fetch_back(q, top - kGtsvChunk, nr, act, c, U, G);
        const GtsvSmem& cur = sm[cb];
        const int n = (int)((top + 1 < kGtsvChunk) ? (top + 1) : kGtsvChunk);
#pragma unroll 1
        for (int u = 0; u < n; ++u) {
            const long long i = top - u;
            double v = cur.f[u][c];
            v = fma(-cur.b[u], x1, v);
            v = fma(-cur.c[u], x2, v);
            const double xi = v * cur.a[u];
            if (act) X[i * nr + c] = xi;
            x2 = x1;
            x1 = xi;
        }
        cb ^= 1;
        gtsv_park(sm[cb], q, c);
        __syncwarp();
    }
}

size_t btri_direct_smem(int m, int nr) { return sizeof(double) * ((size_t)(2 * m) * (3 * m + nr) + 2 * m); }
cudaError_t launch_btri_direct(int K, int m, int nr, const double* B, const double* D, const double* C,
                               const double* F, double* X, double* keep, long long* status, int level,
                               cudaStream_t s) {
    if (m == 1) {
        k_gtsv<<<1, 32, 0, s>>>(K, nr, B, D, C, F, X, keep, status, level);
        return cudaGetLastError();
    }
    const size_t smem = btri_direct_smem(m, nr);
    if (smem > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(k_btri_direct, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
    }
    k_btri_direct<<<1, 256, smem, s>>>(K, m, nr, B, D, C, F, X, keep, status, level);
    return cudaGetLastError();
}
cudaError_t launch_babd_direct(int Np, int m, int nr, const double* S, const double* R, const double* B0,
                               const double* B1, const double* F, double* X, double* keep, long long* status,
                               int level, cudaStream_t s) {
    const size_t smem = babd_direct_smem(m, nr);
    if (smem > 48 * 1024) {   // per device and cheap: set it whenever it is needed
        cudaError_t e = cudaFuncSetAttribute(k_babd_direct, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
    }
    k_babd_direct<<<1, 256, smem, s>>>(Np, m, nr, S, R, B0, B1, F, X, keep, status, level);
    return cudaGetLastError();
}

}  // namespace bt

namespace bt {

// out[j] (M x M) = [[in[j], 0], [0, tail]] for j < N (in: m x m), tail = I or 0.
__global__ void __launch_bounds__(256) k_pad_blocks(long long N, int m, int M, const double* __restrict__ in,
                                                    double* __restrict__ out, int identity_tail) {
    const long long MM = (long long)M * M;
    const long long total = N * MM;
    for (long long el = (long long)blockIdx.x * blockDim.x + threadIdx.x; el < total;
         el += (long long)gridDim.x * blockDim.x) {
        const long long j = el / MM;
        const int r = (int)((el % MM) / M), c = (int)(el % M);
        double v;
        if (r < m && c < m) v = in[j * m * m + (long long)r * m + c];
        else v = (identity_tail && r == c) ? 1.0 : 0.0;
        out[el] = v;
    }
}

// Right-hand sides [rows][m][nr] <-> [rows][M][nr] (zero padding).
__global__ void __launch_bounds__(256) k_pad_rhs(long long rows, int m, int M, int nr, const double* __restrict__ in,
                                                 double* __restrict__ out) {
    const long long total = rows * M * nr;
    for (long long el = (long long)blockIdx.x * blockDim.x + threadIdx.x; el < total;
         el += (long long)gridDim.x * blockDim.x) {
        const long long j = el / ((long long)M * nr);
        const int r = (int)((el / nr) % M), c = (int)(el % nr);
        out[el] = (r < m) ? in[(j * m + r) * nr + c] : 0.0;
    }
}
__global__ void __launch_bounds__(256) k_unpad_rhs(long long rows, int m, int M, int nr, const double* __restrict__ in,
                                                   double* __restrict__ out) {
    const long long total = rows * m * nr;
    for (long long el = (long long)blockIdx.x * blockDim.x + threadIdx.x; el < total;
         el += (long long)gridDim.x * blockDim.x) {
        const long long j = el / ((long long)m * nr);
        const int r = (int)((el / nr) % m), c = (int)(el % nr);
        out[el] = in[(j * M + r) * nr + c];
    }
}

// Banded matrix (s sub-, r super-diagonals) in band storage band[(r + i - k) * n + k] = A[i][k]
// -> block tridiagonal blocks of order m >= max(s, r), N = ceil(n / m); unknowns beyond n get
// an identity row.
__global__ void __launch_bounds__(256) k_band_to_blocks(long long n, int s, int r, const double* __restrict__ band,
                                                        long long N, int m, double* __restrict__ B,
                                                        double* __restrict__ D, double* __restrict__ C) {
    const long long mm = (long long)m * m;
    const long long total = N * mm;
    for (long long el = (long long)blockIdx.x * blockDim.x + threadIdx.x; el < total;
         el += (long long)gridDim.x * blockDim.x) {
        const long long j = el / mm;
        const int a = (int)((el % mm) / m), b = (int)(el % m);
        const long long i = j * m + a;   // global row
        for (int blk = 0; blk < 3; ++blk) {
            const long long k = (j + blk - 1) * m + b;   // global column in block column j-1, j, j+1
            double v = 0.0;
            if (i < n && k >= 0 && k < n && i - k <= s && k - i <= r) v = band[(long long)(r + i - k) * n + k];
            if (blk == 1 && i >= n && a == b) v = 1.0;
            double* dst = (blk == 0) ? B : (blk == 1) ? D : C;
            dst[el] = v;
        }
    }
}

static unsigned grid_stride(long long total) {
    long long g = (total + 255) / 256;
    if (g > 4096) g = 4096;
    if (g < 1) g = 1;
    return (unsigned)g;
}

cudaError_t launch_pad_blocks(long long N, int m, int M, const double* in, double* out, int identity_tail,
                              cudaStream_t s) {
    if (N <= 0) return cudaSuccess;
    k_pad_blocks<<<grid_stride(N * M * M), 256, 0, s>>>(N, m, M, in, out, identity_tail);
    return cudaGetLastError();
}
cudaError_t launch_pad_rhs(long long rows, int m, int M, int nr, const double* in, double* out, cudaStream_t s) {
    k_pad_rhs<<<grid_stride(rows * M * nr), 256, 0, s>>>(rows, m, M, nr, in, out);
    return cudaGetLastError();
}
cudaError_t launch_unpad_rhs(long long rows, int m, int M, int nr, const double* in, double* out, cudaStream_t s) {
    k_unpad_rhs<<<grid_stride(rows * m * nr), 256, 0, s>>>(rows, m, M, nr, in, out);
    return cudaGetLastError();
}
cudaError_t launch_band_to_blocks(long long n, int s_, int r, const double* band, long long N, int m, double* B,
                                  double* D, double* C, cudaStream_t s) {
    k_band_to_blocks<<<grid_stride(N * m * m), 256, 0, s>>>(n, s_, r, band, N, m, B, D, C);
    return cudaGetLastError();
}

}  // namespace bt

namespace bt {
namespace {
// y = rcp(x) elementwise: the FP64 reciprocal every FP64 pivot step uses.
__global__ void __launch_bounds__(256) k_rcp(long long n, const double* __restrict__ x, double* __restrict__ y) {
    for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (long long)gridDim.x * blockDim.x)
        y[e] = rcp(x[e]);
}
}  // namespace
}  // namespace bt

extern "C" bt_status bt_device_rcp(int64_t n, const double* x, double* y, void* stream) {
    if (n < 0 || (n > 0 && (x == nullptr || y == nullptr))) return BT_ERR_INVALID;
    if (n == 0) return BT_OK;
    long long blocks = (n + 255) / 256;
    if (blocks > 8192) blocks = 8192;
    bt::k_rcp<<<(unsigned)blocks, 256, 0, (cudaStream_t)stream>>>(n, x, y);
    return cudaGetLastError() == cudaSuccess ? BT_OK : BT_ERR_CUDA;
}
