// Parareal (Sec. 4): the iterative solution of the reduced system (redsys) of
// the parallel IVP solver (Sec. 3) by the splitting F = (F - G) + G, for
// y' = L y + g0 + t g1 with L tridiagonal.  The fine propagation of all p
// coarse intervals is one sequence of nfine tridiagonal solves with p
// right-hand sides (the intervals advance together); the coarse correction
// sweep is sequential over the intervals.  Both tridiagonal operators are
// factored once by the partition-method plans of bt.h.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>
#include <vector>

#include "../../include/bt.h"
#include "../../include/bt_ivp.h"

namespace {

constexpr int kThreads = 256;

inline unsigned grid_for(long long n) { return (unsigned)std::max<long long>(1, (n + kThreads - 1) / kThreads); }

// I - a L as blocks of order 1: B = -a dl, D = 1 - a d, C = -a du.
__global__ void k_ivp_shift(long long n, double a, const double* __restrict__ dl, const double* __restrict__ d,
                            const double* __restrict__ du, double* B, double* D, double* C) {
    const long long j = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= n) return;
    B[j] = (j > 0) ? -a * dl[j] : 0.0;
    D[j] = 1.0 - a * d[j];
    C[j] = (j + 1 < n) ? -a * du[j] : 0.0;
}

// Y[j][i] = U[i][j] for the p interval start values (U: [p+1][n], Y: [n][p]).
__global__ void k_ivp_gather(long long n, int p, const double* __restrict__ U, double* __restrict__ Y) {
    const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= n * p) return;
    const long long j = idx / p;
    const int i = (int)(idx % p);
    Y[idx] = U[(long long)i * n + j];
}

// Right-hand side of trapezoidal step `step` of every interval i (start time
// i H): R = Y + h/2 L Y + h/2 (g(t) + g(t + h)), t = i H + step h.
__global__ void k_ivp_trap_rhs(long long n, int p, double h, double H, int step, const double* __restrict__ dl,
                               const double* __restrict__ d, const double* __restrict__ du,
                               const double* __restrict__ g0, const double* __restrict__ g1,
                               const double* __restrict__ Y, double* __restrict__ R) {
    const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= n * p) return;
    const long long j = idx / p;
    const int i = (int)(idx % p);
    const double y = Y[idx];
    double Ly = d[j] * y;
    if (j > 0) Ly += dl[j] * Y[idx - p];
    if (j + 1 < n) Ly += du[j] * Y[idx + p];
    const double t = i * H + step * h;
    double g = 2.0 * g0[j];
    if (g1) g += g1[j] * (2.0 * t + h);
    R[idx] = y + 0.5 * h * Ly + 0.5 * h * g;
}

// Right-hand side of a backward Euler step ending at t1: r = y + hc g(t1).
__global__ void k_ivp_be_rhs(long long n, double hc, double t1, const double* __restrict__ g0,
                             const double* __restrict__ g1, const double* __restrict__ y, double* __restrict__ r) {
    const long long j = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= n) return;
    double g = g0[j];
    if (g1) g += g1[j] * t1;
    r[j] = y[j] + hc * g;
}

// Parareal correction of interval i: U_{i+1} = G_new + F_i U_i^(k) - G_old.
__global__ void k_ivp_correct(long long n, int p, int i, const double* __restrict__ Gnew,
                              const double* __restrict__ Fv, const double* __restrict__ Gold,
                              double* __restrict__ Unext) {
    const long long j = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= n) return;
    Unext[j] = (Gnew[j] + Fv[j * p + i]) - Gold[j];
}

// out[0] = max |a - b|, out[1] = max |a| as bit patterns (integer atomicMax).
__global__ void k_ivp_maxdiff(long long len, const double* __restrict__ a, const double* __restrict__ b,
                              unsigned long long* out) {
    unsigned long long dmax = 0ull, amax = 0ull;
    for (long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x; k < len;
         k += (long long)gridDim.x * blockDim.x) {
        const unsigned long long dk = (unsigned long long)__double_as_longlong(fabs(a[k] - b[k]));
        const unsigned long long ak = (unsigned long long)__double_as_longlong(a[k]) & 0x7fffffffffffffffull;
        dmax = dk > dmax ? dk : dmax;
        amax = ak > amax ? ak : amax;
    }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
        const unsigned long long d2 = __shfl_xor_sync(0xffffffffu, dmax, off);
        const unsigned long long a2 = __shfl_xor_sync(0xffffffffu, amax, off);
        dmax = d2 > dmax ? d2 : dmax;
        amax = a2 > amax ? a2 : amax;
    }
    if ((threadIdx.x & 31) == 0) {
        atomicMax(out, dmax);
        atomicMax(out + 1, amax);
    }
}

struct Work {
    std::vector<void*> bufs;
    bt_plan pf = nullptr, pc = nullptr;
    ~Work() {
        if (pf) bt_plan_destroy(pf);
        if (pc) bt_plan_destroy(pc);
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

extern "C" bt_status ivp_parareal(int64_t n, const double* dl, const double* d, const double* du, const double* g0,
                                  const double* g1, const double* y0, double T, int p, int nfine, int ncoarse,
                                  int kmax, double tol, double* U, double* hist, int* iters_out, void* stream) {
    if (iters_out) *iters_out = 0;
    if (n < 1 || !dl || !d || !du || !g0 || !y0 || !U || p < 1 || p > 32 || nfine < 1 || ncoarse < 1 || kmax < 0 ||
        kmax > p || !(T > 0.0) || !(tol >= 0.0))
        return BT_ERR_INVALID;
    cudaStream_t s = (cudaStream_t)stream;
    const double H = T / p, h = H / nfine, hc = H / ncoarse;
    const size_t nn = (size_t)n, np = nn * p;
    Work w;
    cudaError_t e = cudaSuccess;
    double* Bf = w.take(nn, e);
    double* Df = w.take(nn, e);
    double* Cf = w.take(nn, e);
    double* Bc = w.take(nn, e);
    double* Dc = w.take(nn, e);
    double* Cc = w.take(nn, e);
    double* Y = w.take(np, e);       // [n][p] fine states
    double* R = w.take(np, e);       // [n][p] right-hand sides
    double* Un = w.take(nn * (p + 1), e);   // next iterate
    double* Gold = w.take(nn * p, e);       // G_i U_i^(k), [p][n]
    double* r = w.take(nn, e);
    double* gn = w.take(nn, e);
    unsigned long long* red = (unsigned long long*)w.take(2, e);
    if (e != cudaSuccess) return cuda_status(e);
    k_ivp_shift<<<grid_for(n), kThreads, 0, s>>>(n, 0.5 * h, dl, d, du, Bf, Df, Cf);
    k_ivp_shift<<<grid_for(n), kThreads, 0, s>>>(n, hc, dl, d, du, Bc, Dc, Cc);
    e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_status(e);
    bt_status st = bt_plan_create(&w.pf, n, 1, p, BT_FP64, 0, stream);
    if (st == BT_OK) st = bt_plan_create(&w.pc, n, 1, 1, BT_FP64, 0, stream);
    if (st == BT_OK) st = bt_factor(w.pf, Bf, Df, Cf);
    if (st == BT_OK) st = bt_factor(w.pc, Bc, Dc, Cc);
    if (st != BT_OK) return st;

    // coarse propagator G_i applied to `in` (interval i), result in `out`
    // (each step: r = y + hc g(t1), then solve (I - hc L) out = r)
    auto coarse = [&](int i, const double* in, double* out) -> bt_status {
        const double* cur = in;
        for (int k = 0; k < ncoarse; ++k) {
            const double t1 = i * H + (k + 1) * hc;
            k_ivp_be_rhs<<<grid_for(n), kThreads, 0, s>>>(n, hc, t1, g0, g1, cur, r);
            bt_status q = bt_solve(w.pc, r, out, 1);
            if (q != BT_OK) return q;
            cur = out;
        }
        return BT_OK;
    };
    const size_t vbytes = sizeof(double) * nn;
    // k = 0: the sequential coarse sweep
    e = cudaMemcpyAsync(U, y0, vbytes, cudaMemcpyDeviceToDevice, s);
    if (e != cudaSuccess) return cuda_status(e);
    for (int i = 0; i < p && st == BT_OK; ++i) {
        st = coarse(i, U + i * nn, U + (i + 1) * nn);
        if (st == BT_OK)
            e = cudaMemcpyAsync(Gold + i * nn, U + (i + 1) * nn, vbytes, cudaMemcpyDeviceToDevice, s);
        if (e != cudaSuccess) return cuda_status(e);
    }
    if (st != BT_OK) return st;
    if (hist) {
        e = cudaMemcpyAsync(hist, U, vbytes * (p + 1), cudaMemcpyDeviceToDevice, s);
        if (e != cudaSuccess) return cuda_status(e);
    }
    bool converged = (kmax == 0);
    int it = 0;
    for (int k = 0; k < kmax; ++k) {
        // fine propagation of every interval from U^(k): Y <- F_i U_i (column i)
        k_ivp_gather<<<grid_for((long long)np), kThreads, 0, s>>>(n, p, U, Y);
        for (int step = 0; step < nfine && st == BT_OK; ++step) {
            k_ivp_trap_rhs<<<grid_for((long long)np), kThreads, 0, s>>>(n, p, h, H, step, dl, d, du, g0, g1, Y, R);
            st = bt_solve(w.pf, R, Y, p);
        }
        if (st != BT_OK) return st;
        // sequential correction sweep
        e = cudaMemcpyAsync(Un, y0, vbytes, cudaMemcpyDeviceToDevice, s);
        for (int i = 0; i < p && st == BT_OK && e == cudaSuccess; ++i) {
            st = coarse(i, Un + i * nn, gn);   // G_i U_i^(k+1)
            if (st != BT_OK) break;
            k_ivp_correct<<<grid_for(n), kThreads, 0, s>>>(n, p, i, gn, Y, Gold + i * nn, Un + (i + 1) * nn);
            e = cudaMemcpyAsync(Gold + i * nn, gn, vbytes, cudaMemcpyDeviceToDevice, s);
        }
        if (st != BT_OK) return st;
        if (e != cudaSuccess) return cuda_status(e);
        // convergence test on the change of the iterate
        unsigned long long hr[2] = {0ull, 0ull};
        e = cudaMemsetAsync(red, 0, 2 * sizeof(unsigned long long), s);
        if (e == cudaSuccess) {
            k_ivp_maxdiff<<<std::min<unsigned>(grid_for((long long)(nn * (p + 1))), 1024u), kThreads, 0, s>>>(
                (long long)(nn * (p + 1)), Un, U, red);
            e = cudaMemcpyAsync(hr, red, sizeof(hr), cudaMemcpyDeviceToHost, s);
        }
        if (e == cudaSuccess) e = cudaMemcpyAsync(U, Un, vbytes * (p + 1), cudaMemcpyDeviceToDevice, s);
        if (e == cudaSuccess && hist)
            e = cudaMemcpyAsync(hist + (size_t)(k + 1) * (p + 1) * nn, Un, vbytes * (p + 1), cudaMemcpyDeviceToDevice,
                                s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) return cuda_status(e);
        it = k + 1;
        double dmax, amax;
        static_assert(sizeof(double) == sizeof(unsigned long long), "");
        std::memcpy(&dmax, &hr[0], sizeof(double));
        std::memcpy(&amax, &hr[1], sizeof(double));
        if (dmax <= tol * amax) {
            converged = true;
            break;
        }
    }
    if (iters_out) *iters_out = it;
    e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return cuda_status(e);
    st = bt_sync(w.pf);
    if (st == BT_OK) st = bt_sync(w.pc);
    if (st != BT_OK) return st;
    return converged ? BT_OK : BT_ERR_NOT_CONVERGED;
}
