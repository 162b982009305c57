// Parallel IVP solver with a block Boundary Value Method as the local method
// (Sec. 3: Eqs. (M_iy_i), (My), (D), (redsys)/(recur) and the parallel updates
// (pups)) for y' = L y + g(t), L constant (m x m), y(0) = y0, on p coarse
// intervals of N steps each (h = T / (p N)).
//
// Local method: the generalized Adams BVM with k = 2 (order 3) as main
// formula, y_n - y_{n-1} = h (b0 f_{n-1} + b1 f_n + b2 f_{n+1}), with the
// trapezoidal rule as the final formula at n = N; each M_i is then block
// tridiagonal, and with constant L and equal steps it is the same matrix M
// for every interval.  The algorithm:
//   (D)       M [z_1 ... z_p | w] = [g_1 ... g_p | v]   -- one factorization
//             of M by the partition method, all intervals' right-hand sides
//             (and the propagator w = M^{-1} v) solved in parallel;
//   (redsys)  y_{0,1} = y0, y_{0,i+1} = z_{N,i} + w_N y_{0,i}  (p steps);
//   (pups)    y_i = z_i + w y_{0,i}, every interval and row in parallel.
#include <cuda_runtime.h>

#include <algorithm>
#include <vector>

#include "../../include/bt.h"
#include "../../include/bt_ivp.h"

namespace {

constexpr int kThreads = 256;
constexpr int kCols = 32;   // right-hand sides per solve (the plans' nrhs limit)

inline unsigned grid_for(long long n) { return (unsigned)std::max<long long>(1, (n + kThreads - 1) / kThreads); }

struct Coef {
    double b0, b1, b2;
};

// Coefficients of the main formula from its order conditions: exactness on
// y = t^q, q = 1..3, with nodes 0, 1, 2 (h = 1):  sum_j b_j q j^(q-1) = 1.
// The 3 x 3 system [[1,1,1],[0,2,4],[0,3,12]] b = [1,1,1] by Cramer's rule.
Coef gam3() {
    const double A[3][3] = {{1, 1, 1}, {0, 2, 4}, {0, 3, 12}};
    auto det = [](const double M[3][3]) {
        return M[0][0] * (M[1][1] * M[2][2] - M[1][2] * M[2][1]) - M[0][1] * (M[1][0] * M[2][2] - M[1][2] * M[2][0]) +
               M[0][2] * (M[1][0] * M[2][1] - M[1][1] * M[2][0]);
    };
    const double d = det(A);
    double b[3];
    for (int c = 0; c < 3; ++c) {
        double Mc[3][3];
        for (int r = 0; r < 3; ++r)
            for (int k = 0; k < 3; ++k) Mc[r][k] = (k == c) ? 1.0 : A[r][k];
        b[c] = det(Mc) / d;
    }
    return {b[0], b[1], b[2]};
}

// Block rows of M: rows n < N - 1 the main formula, row N - 1 the final one.
__global__ void k_bvm_blocks(long long N, int m, double h, Coef cf, const double* __restrict__ L,
                             double* __restrict__ B, double* __restrict__ D, double* __restrict__ C) {
    const long long mm = (long long)m * m;
    const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= N * mm) return;
    const long long n = e / mm;
    const int rc = (int)(e % mm), r = rc / m, c = rc % m;
    const double l = L[rc], id = (r == c) ? 1.0 : 0.0;
    if (n < N - 1) {
        B[e] = -(id + h * cf.b0 * l);
        D[e] = id - h * cf.b1 * l;
        C[e] = -h * cf.b2 * l;
    } else {
        B[e] = -(id + 0.5 * h * l);
        D[e] = id - 0.5 * h * l;
        C[e] = 0.0;
    }
}

// V [N m][m]: the coupling of block row 1 to the interval's initial value,
// v = -B_1 (I + h b0 L, or I + h/2 L when the interval has one step), zero below.
__global__ void k_bvm_v(long long N, int m, double h, Coef cf, const double* __restrict__ L, double* __restrict__ V) {
    const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= N * m * m) return;
    const long long row = e / m;
    const int c = (int)(e % m);
    if (row >= m) {
        V[e] = 0.0;
        return;
    }
    const int r = (int)row;
    const double a = (N > 1) ? h * cf.b0 : 0.5 * h;
    V[e] = ((r == c) ? 1.0 : 0.0) + a * L[r * m + c];
}

// Right-hand sides of intervals i0 .. i0 + cols - 1 as the columns of R [N m][cols].
__global__ void k_bvm_rhs(long long N, int m, int cols, long long i0, double h, Coef cf, const double* __restrict__ G,
                          double* __restrict__ R) {
    const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= N * m * cols) return;
    const int col = (int)(e % cols);
    const long long row = e / cols;
    const long long n = row / m;
    const int r = (int)(row % m);
    const long long k = (i0 + col) * N + n;   // global grid index of the interval's point n
    double v;
    if (n < N - 1)
        v = h * (cf.b0 * G[k * m + r] + cf.b1 * G[(k + 1) * m + r] + cf.b2 * G[(k + 2) * m + r]);
    else
        v = 0.5 * h * (G[k * m + r] + G[(k + 1) * m + r]);
    R[e] = v;
}

// Z [p][N][m] <- the solution columns of a chunk, Zc [N m][cols].
__global__ void k_bvm_store(long long N, int m, int cols, long long i0, const double* __restrict__ Zc,
                            double* __restrict__ Z) {
    const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= N * m * cols) return;
    const int col = (int)(e % cols);
    const long long row = e / cols;
    Z[(i0 + col) * N * m + row] = Zc[e];
}

// (redsys): y_{0,1} = y0, y_{0,i+1} = z_{N,i} + w_N y_{0,i} (one CTA; thread r
// owns entry r; four partial sums per dot product).
__global__ void k_bvm_recur(long long p, long long N, int m, const double* __restrict__ Z,
                            const double* __restrict__ W, const double* __restrict__ y0, double* __restrict__ Y0) {
    __shared__ double cur[32];
    const int r = threadIdx.x;
    if (r < m) {
        cur[r] = y0[r];
        Y0[r] = y0[r];
    }
    __syncthreads();
    const double* WN = W + (N - 1) * m * m;
    for (long long i = 0; i < p; ++i) {
        double nxt = 0.0;
        if (r < m) {
            double s[4] = {0.0, 0.0, 0.0, 0.0};
            for (int k = 0; k < m; ++k) s[k & 3] = fma(WN[r * m + k], cur[k], s[k & 3]);
            nxt = Z[(i * N + N - 1) * m + r] + ((s[0] + s[1]) + (s[2] + s[3]));
        }
        __syncthreads();
        if (r < m) {
            cur[r] = nxt;
            Y0[(i + 1) * m + r] = nxt;
        }
        __syncthreads();
    }
}

// (pups): Y[i N + n + 1] = z_{n,i} + w_n y_{0,i}; Y[0] = y0.
__global__ void k_bvm_update(long long p, long long N, int m, const double* __restrict__ Z,
                             const double* __restrict__ W, const double* __restrict__ Y0, double* __restrict__ Y) {
    const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const long long tot = p * N * m;
    if (e < m) Y[e] = Y0[e];
    if (e >= tot) return;
    const long long i = e / (N * m), rem = e % (N * m), n = rem / m;
    const int r = (int)(rem % m);
    const double* Wn = W + n * m * m + (long long)r * m;
    const double* y0i = Y0 + i * m;
    double s0 = 0.0, s1 = 0.0;
    for (int k = 0; k + 1 < m; k += 2) {
        s0 = fma(Wn[k], y0i[k], s0);
        s1 = fma(Wn[k + 1], y0i[k + 1], s1);
    }
    if (m & 1) s0 = fma(Wn[m - 1], y0i[m - 1], s0);
    Y[(i * N + n + 1) * m + r] = Z[e] + (s0 + s1);
}

struct Work {
    std::vector<void*> bufs;
    bt_plan plan = nullptr;
    ~Work() {
        if (plan) bt_plan_destroy(plan);
        for (void* b : bufs) cudaFree(b);
    }
    double* take(size_t count, cudaError_t& e) {
        void* q = nullptr;
        if (e == cudaSuccess) e = cudaMalloc(&q, sizeof(double) * std::max<size_t>(count, 1));
        if (e == cudaSuccess) bufs.push_back(q);
        return (double*)q;
    }
};

bt_status cuda_status(cudaError_t e) {
    if (e == cudaSuccess) return BT_OK;
    return e == cudaErrorMemoryAllocation ? BT_ERR_NOMEM : BT_ERR_CUDA;
}

}  // namespace

extern "C" bt_status ivp_bvm(int m, int64_t p, int64_t N, double T, const double* L, const double* y0,
                             const double* G, double* Y, void* stream) {
    if (m < 1 || m > 32 || p < 1 || N < 1 || !(T > 0.0) || !L || !y0 || !G || !Y) return BT_ERR_INVALID;
    cudaStream_t s = (cudaStream_t)stream;
    const double h = T / ((double)p * (double)N);
    const Coef cf = gam3();
    const long long mm = (long long)m * m;
    Work w;
    cudaError_t e = cudaSuccess;
    double* B = w.take(N * mm, e);
    double* D = w.take(N * mm, e);
    double* C = w.take(N * mm, e);
    double* V = w.take(N * mm, e);
    double* W = w.take(N * mm, e);
    double* R = w.take(N * m * kCols, e);
    double* Zc = w.take(N * m * kCols, e);
    double* Z = w.take((size_t)p * N * m, e);
    double* Y0 = w.take((size_t)(p + 1) * m, e);
    if (e != cudaSuccess) return cuda_status(e);
    k_bvm_blocks<<<grid_for(N * mm), kThreads, 0, s>>>(N, m, h, cf, L, B, D, C);
    k_bvm_v<<<grid_for(N * mm), kThreads, 0, s>>>(N, m, h, cf, L, V);
    e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_status(e);
    // (D): one factorization of M, then every right-hand side
    bt_status st = bt_plan_create(&w.plan, N, m, kCols, BT_FP64, 0, stream);
    if (st == BT_OK) st = bt_factor(w.plan, B, D, C);
    if (st == BT_OK) st = bt_solve(w.plan, V, W, m);
    for (long long i0 = 0; i0 < p && st == BT_OK; i0 += kCols) {
        const int cols = (int)std::min<long long>(kCols, p - i0);
        k_bvm_rhs<<<grid_for(N * m * cols), kThreads, 0, s>>>(N, m, cols, i0, h, cf, G, R);
        st = bt_solve(w.plan, R, Zc, cols);
        if (st == BT_OK) k_bvm_store<<<grid_for(N * m * cols), kThreads, 0, s>>>(N, m, cols, i0, Zc, Z);
    }
    if (st != BT_OK) return st;
    // (redsys) then (pups)
    k_bvm_recur<<<1, 32, 0, s>>>(p, N, m, Z, W, y0, Y0);
    k_bvm_update<<<grid_for(std::max<long long>(p * N * m, m)), kThreads, 0, s>>>(p, N, m, Z, W, Y0, Y);
    e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return cuda_status(e);
    return bt_sync(w.plan);
}
