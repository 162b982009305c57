// Local QR factorization of the partitions (Sec. 2, N^(i) = Q^(i),
// S^(i) = R^(i)) and its two solve passes; layout and formulas in bt_qr.h.
//
// Factorization, one CTA per partition, block rows top to bottom.  The CTA
// keeps a window of two block rows in shared memory, [row j; row j+1] over
// the block columns (j, j+1, j+2, left separator, identity 2m): the top row
// carries what the previous step left of row j, the bottom row is A's row
// j+1.  m Householder reflections (column c: thread 0's warp forms the
// reflector from rows c..H-1, every thread then updates one column of the
// window) turn the panel [D~_j; B_{j+1}] into [R_jj; 0] and the identity
// columns into Q_j^T.  The top row is then final (R_jj, R_{j,j+1},
// R_{j,j+2}, z_j), the bottom row becomes the next top row.  In the same
// pass the left separator's row is carried along:
//   w_j^T R_jj = c0_j^T - w_{j-1}^T R_{j-1,j} - w_{j-2}^T R_{j-2,j}
// (c0_s = C_{s-1}, zero below) by forward substitution, with the running
// sums -w^T z and -w^T y; at the last local row v^T = B_e R_{e-1,e-1}^{-1}
// and the right separator's entries of T_p follow.
#include <cuda_runtime.h>

#include <algorithm>

#include "bt_device.cuh"
#include "bt_qr.h"

namespace bt {
namespace {

template <int M>
struct QrF {
    static constexpr int H2 = 2 * M;
    static constexpr int NC = 6 * M;                 // window columns
    static constexpr int LD = NC + 1;                // odd stride: column reads hit distinct banks
    static constexpr int T = NC <= 32 ? 32 : ((NC + 31) / 32) * 32;
    static constexpr int MM = M * M;
    static constexpr int MP = M * (M + 1);           // m x m with padded rows
    static constexpr int WIN = H2 * LD;
    // window, reflector, W ring [2], R_{j,j+1} ring [2], R_{j,j+2} ring [2], G, -w^T z, -w^T y, v^T
    static constexpr int DOUBLES = WIN + H2 + 2 * MP + 2 * MM + 2 * MM + MP + MM + MM + MP;
    static constexpr size_t SMEM = sizeof(double) * DOUBLES;
};

// Thread 0's warp: the reflector H = I - tau v v^T (v_c = 1) with
// H x = beta e_c for x = window column c, rows c..H-1 (dlarfg convention:
// beta = -sign(x_c) ||x||, tau = 0 when the rows below c are zero).  Writes
// v to vec, beta and zeros to column c, returns tau (lane 0 reports a zero or
// non-finite R_cc).
template <int M>
__device__ __forceinline__ double qr_reflector(double* w, double* vec, int c, int H, int lane, long long* status,
                                               long long part, long long row) {
    constexpr int LD = QrF<M>::LD;
    double x0 = 0.0, x1 = 0.0;
    const int r0 = c + lane, r1 = c + 32 + lane;
    if (r0 < H) x0 = w[r0 * LD + c];
    if (r1 < H) x1 = w[r1 * LD + c];
    double sc = fmax(fabs(x0), fabs(x1));
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) sc = fmax(sc, __shfl_xor_sync(0xffffffffu, sc, o));
    const double xc = __shfl_sync(0xffffffffu, x0, 0);
    double tau = 0.0, beta = xc;
    bool sub = false;   // rows below c not all zero
    if (sc > 0.0 && !nonfinite(sc)) {
        const double is = 1.0 / sc;
        const double a0 = (r0 > c) ? x0 * is : 0.0, a1 = x1 * is;
        double sig = fma(a0, a0, a1 * a1);
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) sig += __shfl_xor_sync(0xffffffffu, sig, o);
        if (sig > 0.0) {
            sub = true;
            const double xs = xc * is;
            const double nrm = sc * sqrt(fma(xs, xs, sig));
            beta = (xc >= 0.0) ? -nrm : nrm;
            tau = (beta - xc) / beta;
            const double scl = 1.0 / (xc - beta);
            if (r0 > c && r0 < H) vec[r0] = x0 * scl;
            if (r1 < H) vec[r1] = x1 * scl;
        }
    }
    if (lane == 0) {
        vec[c] = 1.0;
        w[c * LD + c] = beta;
        if (nonfinite(sc) || nonfinite(beta)) report(status, ST_NONFINITE, 0, part, row);
        else if (beta == 0.0) report(status, ST_SINGULAR, 0, part, row);
    }
    if (sub) {
        if (r0 > c && r0 < H) w[r0 * LD + c] = 0.0;
        if (r1 < H) w[r1 * LD + c] = 0.0;
    }
    return tau;
}

// Entry (r, k) of the product of two m x m operands: sum_l a[r][l] b[l][k].
template <int M>
__device__ __forceinline__ double dot_rows(const double* a, int lda, const double* b, int ldb, int r, int k) {
    double s0 = 0.0, s1 = 0.0;
#pragma unroll
    for (int l = 0; l + 1 < M; l += 2) {
        s0 = fma(a[r * lda + l], b[l * ldb + k], s0);
        s1 = fma(a[r * lda + l + 1], b[(l + 1) * ldb + k], s1);
    }
    if (M & 1) s0 = fma(a[r * lda + M - 1], b[(M - 1) * ldb + k], s0);
    return s0 + s1;
}

// Row r of X solving X R = G for upper triangular R (forward substitution
// over the columns): X[r][k] = (G[r][k] - sum_{l<k} X[r][l] R[l][k]) / R[k][k].
template <int M>
__device__ __forceinline__ void right_trsm_row(const double* G, int ldg, const double* R, int ldr, double* X, int ldx,
                                               int r) {
    for (int k = 0; k < M; ++k) {
        double acc = G[r * ldg + k];
        for (int l = 0; l < k; ++l) acc = fma(-X[r * ldx + l], R[l * ldr + k], acc);
        X[r * ldx + k] = acc / R[k * ldr + k];
    }
}


__device__ __forceinline__ void qr_cp16(void* dst, const void* src) {
    const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(d), "l"(src) : "memory");
}
__device__ __forceinline__ void qr_cp8(void* dst, const void* src) {
    const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(d), "l"(src) : "memory");
}
__device__ __forceinline__ void qr_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N>
__device__ __forceinline__ void qr_wait() {
    asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory");
}

template <int M>
__global__ void __launch_bounds__(QrF<M>::T) k_qr_factor(QrArgs a) {
    using F = QrF<M>;
    constexpr int LD = F::LD, MM = F::MM, T = F::T, MP1 = M + 1;
    extern __shared__ __align__(16) double sm[];
    double* w = sm;                       // window [2m][LD]
    double* vec = w + F::WIN;             // reflector [2m]
    double* Wr = vec + F::H2;             // w_j^T ring [2][m][m+1]
    double* R1 = Wr + 2 * F::MP;          // R_{j,j+1} ring [2][m][m]
    double* R2 = R1 + 2 * MM;             // R_{j,j+2} ring [2][m][m]
    double* G = R2 + 2 * MM;              // [m][m+1]
    double* Ta = G + F::MP;               // -sum w^T z
    double* Ga = Ta + MM;                 // -w^T y
    double* Vs = Ga + MM;                 // v^T [m][m+1]
    __shared__ double tau_s;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const long long i = blockIdx.x;
    const Part q = part_bounds(0, a.N, a.p, a.base, a.extra, i);
    const long long s = q.s, e = q.e;
    if (e == s) {
        // a partition of one separator row: its couplings enter T_p unchanged
        for (int t = tid; t < MM; t += T) {
            if (q.hasR) {
                a.Dn[i * MM + t] = a.D[e * MM + t];
                a.Bn[i * MM + t] = q.hasL ? a.B[e * MM + t] : 0.0;
                if (q.hasL) a.Cn[(i - 1) * MM + t] = a.C[(s - 1) * MM + t];
            }
            if (q.hasL) a.Ta[i * MM + t] = 0.0;
        }
        return;
    }
    // top row <- block row s: D_s | C_s (column s+1, the right separator when
    // s+1 = e) | 0 | B_s (left separator column)
    for (int t = tid; t < M * 4 * M; t += T) {
        const int r = t / (4 * M), c = t % (4 * M), cb = c / M, cc = c % M;
        double v = 0.0;
        if (cb == 0) v = a.D[s * MM + r * M + cc];
        else if (cb == 1 && (s + 1 < e || q.hasR)) v = a.C[s * MM + r * M + cc];
        else if (cb == 3 && q.hasL) v = a.B[s * MM + r * M + cc];
        w[r * LD + c] = v;
    }
    for (int t = tid; t < MM; t += T) {
        Ta[t] = 0.0;
        Ga[t] = 0.0;
    }
    for (long long j = s; j < e; ++j) {
        const int t = (int)((j - s) & 1);
        const long long tt = j - s;
        const bool last = (j == e - 1);
        const int H = last ? M : 2 * M;
        const int ncol = last ? 5 * M : 6 * M;
        // bottom row <- block row j+1: B_{j+1} | D_{j+1} | C_{j+1} | 0
        if (!last)
            for (int x = tid; x < M * 4 * M; x += T) {
                const int r = x / (4 * M), c = x % (4 * M), cb = c / M, cc = c % M;
                const long long o = (j + 1) * MM + r * M + cc;
                double v = 0.0;
                if (cb == 0) v = a.B[o];
                else if (cb == 1) v = a.D[o];
                else if (cb == 2 && (j + 2 < e || q.hasR)) v = a.C[o];
                w[(M + r) * LD + c] = v;
            }
        for (int x = tid; x < H * 2 * M; x += T) {
            const int r = x / (2 * M), c = x % (2 * M);
            w[r * LD + 4 * M + c] = (r == c) ? 1.0 : 0.0;
        }
        __syncthreads();
        for (int c = 0; c < M; ++c) {
            if (warp == 0) {
                const double tau = qr_reflector<M>(w, vec, c, H, lane, a.status, i, j);
                if (lane == 0) tau_s = tau;
            }
            __syncthreads();
            const double tau = tau_s;
            if (tau != 0.0) {
                for (int col = c + 1 + tid; col < ncol; col += T) {
                    double d0 = 0.0, d1 = 0.0;
                    int r = c;
                    for (; r + 1 < H; r += 2) {
                        d0 = fma(vec[r], w[r * LD + col], d0);
                        d1 = fma(vec[r + 1], w[(r + 1) * LD + col], d1);
                    }
                    if (r < H) d0 = fma(vec[r], w[r * LD + col], d0);
                    const double f = tau * (d0 + d1);
                    for (r = c; r < H; ++r) w[r * LD + col] = fma(-f, vec[r], w[r * LD + col]);
                }
            }
            __syncthreads();
        }
        // the top row is final: R_jj, R_{j,j+1}, R_{j,j+2}, z_j, and Q_j^T
        for (int x = tid; x < MM; x += T) {
            const int r = x / M, k = x % M;
            a.R[(j * 3 + 0) * MM + x] = (k >= r) ? w[r * LD + k] : 0.0;
            a.R[(j * 3 + 1) * MM + x] = w[r * LD + M + k];
            a.R[(j * 3 + 2) * MM + x] = w[r * LD + 2 * M + k];
            a.Z[j * MM + x] = w[r * LD + 3 * M + k];
        }
        for (int x = tid; x < H * H; x += T) {
            const int r = x / H, k = x % H;
            a.Qt[j * 4 * MM + r * 2 * M + k] = w[r * LD + 4 * M + k];
        }
        if (q.hasL) {
            // w_j^T R_jj = c0_j^T - w_{j-1}^T R_{j-1,j} - w_{j-2}^T R_{j-2,j}
            const double* W1 = Wr + (t ^ 1) * F::MP;   // w_{j-1}^T
            double* W2 = Wr + t * F::MP;                // w_{j-2}^T, then w_j^T
            const double* Rp1 = R1 + (t ^ 1) * MM;      // R_{j-1,j}
            const double* Rp2 = R2 + t * MM;            // R_{j-2,j}
            for (int x = tid; x < MM; x += T) {
                const int r = x / M, k = x % M;
                double g = (tt == 0) ? a.C[(s - 1) * MM + x] : 0.0;
                if (tt >= 1) g -= dot_rows<M>(W1, MP1, Rp1, M, r, k);
                if (tt >= 2) g -= dot_rows<M>(W2, MP1, Rp2, M, r, k);
                G[r * MP1 + k] = g;
            }
            __syncthreads();
            if (tid < M) right_trsm_row<M>(G, MP1, w, LD, W2, MP1, tid);
            __syncthreads();
            for (int x = tid; x < MM; x += T) {
                const int r = x / M, k = x % M;
                a.W[j * MM + x] = W2[r * MP1 + k];
                Ta[x] -= dot_rows<M>(W2, MP1, w + 3 * M, LD, r, k);
                if (q.hasR && j == e - 2) Ga[x] -= dot_rows<M>(W2, MP1, w + 2 * M, LD, r, k);
                if (q.hasR && j == e - 1) Ga[x] -= dot_rows<M>(W2, MP1, w + M, LD, r, k);
            }
        }
        for (int x = tid; x < MM; x += T) {
            const int r = x / M, k = x % M;
            R1[t * MM + x] = w[r * LD + M + k];
            R2[t * MM + x] = w[r * LD + 2 * M + k];
        }
        __syncthreads();
        if (!last) {
            // the bottom row becomes the top row, one block column to the left
            for (int x = tid; x < M * 4 * M; x += T) {
                const int r = x / (4 * M), c = x % (4 * M), cb = c / M, cc = c % M;
                const double* bot = w + (M + r) * LD;
                w[r * LD + c] = (cb == 0) ? bot[M + cc] : (cb == 1) ? bot[2 * M + cc] : (cb == 2) ? 0.0 : bot[3 * M + cc];
            }
            __syncthreads();
        }
    }
    // right separator: v^T = B_e R_{e-1,e-1}^{-1}, beta = -v^T z_{e-1}, a_e - v^T y_{e-1}
    if (q.hasR) {
        for (int x = tid; x < MM; x += T) G[(x / M) * MP1 + x % M] = a.B[e * MM + x];
        __syncthreads();
        if (tid < M) right_trsm_row<M>(G, MP1, w, LD, Vs, MP1, tid);
        __syncthreads();
        for (int x = tid; x < MM; x += T) {
            const int r = x / M, k = x % M;
            a.Vb[i * MM + x] = Vs[r * MP1 + k];
            a.Dn[i * MM + x] = a.D[e * MM + x] - dot_rows<M>(Vs, MP1, w + M, LD, r, k);
            a.Bn[i * MM + x] = -dot_rows<M>(Vs, MP1, w + 3 * M, LD, r, k);
        }
    }
    if (q.hasL)
        for (int x = tid; x < MM; x += T) {
            a.Ta[i * MM + x] = Ta[x];
            if (q.hasR) a.Cn[(i - 1) * MM + x] = Ga[x];
        }
}

// v[k] += add[k + off] for k < n (the left partitions' shares of T_p and of
// its right-hand side, with sign).
__global__ void __launch_bounds__(256) k_qr_add(long long n, long long off, double sgn, const double* __restrict__ add,
                                                double* __restrict__ v) {
    for (long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x; k < n; k += (long long)gridDim.x * blockDim.x)
        v[k] = fma(sgn, add[k + off], v[k]);
}

constexpr int kQrSolveThreads = 128;

template <int M>
size_t qr_fwd_smem(int nr) {
    return sizeof(double) * (10 * M * M + 7 * M * nr);
}
template <int M>
size_t qr_bwd_smem(int nr) {
    return sizeof(double) * (8 * M * M + 7 * M * nr);
}

// Forward pass of one partition, top to bottom: [u_j; u~_{j+1}] =
// Q_j^T [u~_j; f_{j+1}] (u~_s = f_s), u_j -> X[j]; the left separator's
// share sum_j w_j^T u_j -> Tf[i]; the right separator's right-hand side
// f_e - v^T u_{e-1} -> Fn[i].  Q_j^T, w_j^T and f_{j+1} of the next row are
// copied into shared memory (cp.async) while the current row is applied.
template <int M>
__global__ void __launch_bounds__(kQrSolveThreads) k_qr_fwd(QrArgs a) {
    constexpr int MM = M * M, Q4 = 4 * MM, T = kQrSolveThreads;
    const int nr = a.nr, mn = M * nr;
    extern __shared__ __align__(16) double sm[];
    double* Qs = sm;                 // [2][4mm] Q_j^T
    double* Ws = Qs + 2 * Q4;        // [2][mm]  w_j^T
    double* Fs = Ws + 2 * MM;        // [2][m nr] f_{j+1}
    double* In = Fs + 2 * mn;        // [2m][nr]
    double* Out = In + 2 * mn;       // [2m][nr]
    double* Tf = Out + 2 * mn;       // [m][nr]
    const int tid = threadIdx.x;
    const long long i = blockIdx.x;
    const Part q = part_bounds(0, a.N, a.p, a.base, a.extra, i);
    const long long s = q.s, e = q.e;
    const long long rowv = mn;
    if (e == s) {
        for (int x = tid; x < mn; x += T) {
            if (q.hasR) a.Fn[i * mn + x] = a.F[e * rowv + x];
            if (q.hasL) a.Tf[i * mn + x] = 0.0;
        }
        return;
    }
    auto stage = [&](long long j, int b) {
        const double* qs = a.Qt + j * Q4;
        for (int c = tid; c < Q4 / 2; c += T) qr_cp16(Qs + b * Q4 + 2 * c, qs + 2 * c);
        if (q.hasL)
            for (int c = tid; c < MM; c += T) qr_cp8(Ws + b * MM + c, a.W + j * MM + c);
        if (j + 1 < e)
            for (int c = tid; c < mn; c += T) qr_cp8(Fs + b * mn + c, a.F + (j + 1) * rowv + c);
        qr_commit();
    };
    for (int x = tid; x < mn; x += T) {
        In[x] = a.F[s * rowv + x];
        Tf[x] = 0.0;
    }
    stage(s, 0);
    for (long long j = s; j < e; ++j) {
        const int b = (int)((j - s) & 1);
        const bool last = (j == e - 1);
        const int H = last ? M : 2 * M;
        if (!last) {
            stage(j + 1, b ^ 1);
            qr_wait<1>();
        } else {
            qr_wait<0>();
        }
        __syncthreads();
        if (!last)
            for (int x = tid; x < mn; x += T) In[mn + x] = Fs[b * mn + x];
        __syncthreads();
        const double* Qj = Qs + b * Q4;
        for (int o = tid; o < H * nr; o += T) {
            const int r = o / nr, c = o % nr;
            double s0 = 0.0, s1 = 0.0;
            int k = 0;
            for (; k + 1 < H; k += 2) {
                s0 = fma(Qj[r * 2 * M + k], In[k * nr + c], s0);
                s1 = fma(Qj[r * 2 * M + k + 1], In[(k + 1) * nr + c], s1);
            }
            if (k < H) s0 = fma(Qj[r * 2 * M + k], In[k * nr + c], s0);
            Out[o] = s0 + s1;
        }
        __syncthreads();
        for (int x = tid; x < mn; x += T) {
            const int r = x / nr, c = x % nr;
            a.X[j * rowv + x] = Out[x];
            if (q.hasL) {
                const double* wr = Ws + b * MM + r * M;
                double acc = Tf[x];
#pragma unroll
                for (int l = 0; l < M; ++l) acc = fma(wr[l], Out[l * nr + c], acc);
                Tf[x] = acc;
            }
            if (!last) In[x] = Out[mn + x];
        }
        __syncthreads();
    }
    for (int x = tid; x < mn; x += T) {
        const int r = x / nr, c = x % nr;
        if (q.hasR) {
            double acc = a.F[e * rowv + x];
            const double* vr = a.Vb + i * MM + r * M;
#pragma unroll
            for (int l = 0; l < M; ++l) acc = fma(-vr[l], Out[l * nr + c], acc);
            a.Fn[i * mn + x] = acc;
        }
        if (q.hasL) a.Tf[i * mn + x] = Tf[x];
    }
}

// Back substitution of one partition, bottom to top:
//   R_jj x_j = u_j - z_j x_L - R_{j,j+1} x_{j+1} - R_{j,j+2} x_{j+2}
// with x_e = the right separator's value and x_{e+1} = 0; the separator rows
// of X take the reduced solution.  The triangular solve: one warp per
// right-hand-side column, lane r holding row r.
template <int M>
__global__ void __launch_bounds__(kQrSolveThreads) k_qr_bwd(QrArgs a) {
    constexpr int MM = M * M, T = kQrSolveThreads;
    const int nr = a.nr, mn = M * nr;
    extern __shared__ __align__(16) double sm[];
    double* Rs = sm;                 // [2][4][mm]: R_jj, R_{j,j+1}, R_{j,j+2}, z_j
    double* Us = Rs + 8 * MM;        // [2][m nr] u_j
    double* Xr = Us + 2 * mn;        // [3][m nr] x_j by j mod 3
    double* XL = Xr + 3 * mn;        // [m nr] left separator
    double* Ts = XL + mn;            // [m nr]
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const long long i = blockIdx.x;
    const Part q = part_bounds(0, a.N, a.p, a.base, a.extra, i);
    const long long s = q.s, e = q.e;
    const long long rowv = mn;
    for (int x = tid; x < mn; x += T) {
        const double xr = q.hasR ? a.Xn[i * mn + x] : 0.0;
        if (q.hasR) a.X[e * rowv + x] = xr;
        Xr[(int)(e % 3) * mn + x] = xr;
        Xr[(int)((e + 1) % 3) * mn + x] = 0.0;
        XL[x] = q.hasL ? a.Xn[(i - 1) * mn + x] : 0.0;
    }
    if (e == s) return;
    auto stage = [&](long long j, int b) {
        double* d = Rs + b * 4 * MM;
        if (M >= 2) {
            for (int c = tid; c < 3 * MM / 2; c += T) qr_cp16(d + 2 * c, a.R + j * 3 * MM + 2 * c);
            for (int c = tid; c < MM / 2; c += T) qr_cp16(d + 3 * MM + 2 * c, a.Z + j * MM + 2 * c);
        } else {
            for (int c = tid; c < 3 * MM; c += T) qr_cp8(d + c, a.R + j * 3 * MM + c);
            for (int c = tid; c < MM; c += T) qr_cp8(d + 3 * MM + c, a.Z + j * MM + c);
        }
        for (int c = tid; c < mn; c += T) qr_cp8(Us + b * mn + c, a.X + j * rowv + c);
        qr_commit();
    };
    stage(e - 1, 0);
    for (long long j = e - 1; j >= s; --j) {
        const int b = (int)((e - 1 - j) & 1);
        if (j > s) {
            stage(j - 1, b ^ 1);
            qr_wait<1>();
        } else {
            qr_wait<0>();
        }
        __syncthreads();
        const double* R0 = Rs + b * 4 * MM;
        const double* R1 = R0 + MM;
        const double* R2 = R0 + 2 * MM;
        const double* Zj = R0 + 3 * MM;
        const double* x1 = Xr + (int)((j + 1) % 3) * mn;
        const double* x2 = Xr + (int)((j + 2) % 3) * mn;
        for (int x = tid; x < mn; x += T) {
            const int r = x / nr, c = x % nr;
            double a0 = Us[b * mn + x], a1 = 0.0;
#pragma unroll
            for (int l = 0; l < M; ++l) {
                a0 = fma(-Zj[r * M + l], XL[l * nr + c], a0);
                a1 = fma(-R1[r * M + l], x1[l * nr + c], a1);
                a0 = fma(-R2[r * M + l], x2[l * nr + c], a0);
            }
            Ts[x] = a0 + a1;
        }
        __syncthreads();
        double* xj = Xr + (int)(j % 3) * mn;
        const double rd = (lane < M) ? 1.0 / R0[lane * M + lane] : 0.0;
        for (int c = warp; c < nr; c += T / 32) {
            double tr = (lane < M) ? Ts[lane * nr + c] : 0.0, xr = 0.0;
            for (int k = M - 1; k >= 0; --k) {
                if (lane == k) xr = tr * rd;
                const double xk = __shfl_sync(0xffffffffu, xr, k);
                if (lane < k) tr = fma(-R0[lane * M + k], xk, tr);
            }
            if (lane < M) {
                xj[lane * nr + c] = xr;
                a.X[j * rowv + lane * nr + c] = xr;
            }
        }
        __syncthreads();
    }
}

template <int M>
cudaError_t set_smem() {
    cudaError_t e = cudaFuncSetAttribute(k_qr_factor<M>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)QrF<M>::SMEM);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_qr_fwd<M>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)qr_fwd_smem<M>(32));
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_qr_bwd<M>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)qr_bwd_smem<M>(32));
    return e;
}

unsigned add_grid(long long n) { return (unsigned)std::max<long long>(1, std::min<long long>((n + 255) / 256, 1216)); }

template <int M>
cudaError_t factor_m(const QrArgs& a, cudaStream_t s) {
    k_qr_factor<M><<<(unsigned)a.p, QrF<M>::T, QrF<M>::SMEM, s>>>(a);
    cudaError_t e = cudaGetLastError();
    const long long n = (a.p - 1) * (long long)M * M;
    if (e == cudaSuccess && n > 0) {
        k_qr_add<<<add_grid(n), 256, 0, s>>>(n, (long long)M * M, 1.0, a.Ta, a.Dn);
        e = cudaGetLastError();
    }
    return e;
}
template <int M>
cudaError_t fwd_m(const QrArgs& a, cudaStream_t s) {
    k_qr_fwd<M><<<(unsigned)a.p, kQrSolveThreads, qr_fwd_smem<M>(a.nr), s>>>(a);
    cudaError_t e = cudaGetLastError();
    const long long n = (a.p - 1) * (long long)M * a.nr;
    if (e == cudaSuccess && n > 0) {
        k_qr_add<<<add_grid(n), 256, 0, s>>>(n, (long long)M * a.nr, -1.0, a.Tf, a.Fn);
        e = cudaGetLastError();
    }
    return e;
}
template <int M>
cudaError_t bwd_m(const QrArgs& a, cudaStream_t s) {
    k_qr_bwd<M><<<(unsigned)a.p, kQrSolveThreads, qr_bwd_smem<M>(a.nr), s>>>(a);
    return cudaGetLastError();
}

}  // namespace

#define BT_QR_DISPATCH(fn, m, ...)                     \
    switch (m) {                                      \
        case 1: return fn<1>(__VA_ARGS__);            \
        case 2: return fn<2>(__VA_ARGS__);            \
        case 4: return fn<4>(__VA_ARGS__);            \
        case 8: return fn<8>(__VA_ARGS__);            \
        case 16: return fn<16>(__VA_ARGS__);          \
        case 32: return fn<32>(__VA_ARGS__);          \
        default: return cudaErrorInvalidValue;        \
    }

cudaError_t qr_prepare(int m) { BT_QR_DISPATCH(set_smem, m) }
cudaError_t launch_qr_factor(const QrArgs& a, cudaStream_t s) {
    if (a.p < 1 || a.nr < 1 || a.nr > 32) return cudaErrorInvalidValue;
    BT_QR_DISPATCH(factor_m, a.m, a, s)
}
cudaError_t launch_qr_solve_fwd(const QrArgs& a, cudaStream_t s) {
    if (a.p < 1 || a.nr < 1 || a.nr > 32) return cudaErrorInvalidValue;
    BT_QR_DISPATCH(fwd_m, a.m, a, s)
}
cudaError_t launch_qr_solve_bwd(const QrArgs& a, cudaStream_t s) {
    if (a.p < 1 || a.nr < 1 || a.nr > 32) return cudaErrorInvalidValue;
    BT_QR_DISPATCH(bwd_m, a.m, a, s)
}

}  // namespace bt
