// Block tridiagonal matrices with corner blocks (Sec. 2, Eqs. (parpart1),
// (redmatr1)); the method is described in include/bt_pbt.h: the end rows are
// separators, the rows between them an inner partition-method plan, and the
// reduced system is closed by the 2m x 2m Schur complement onto the end
// separators.
#include <cuda_runtime.h>

#include <algorithm>
#include <new>

#include "../../include/bt.h"
#include "../../include/bt_pbt.h"

struct pbt_plan_s {
    long long N = 0;
    int m = 0, nrhs_max = 0;
    cudaStream_t stream = nullptr;
    bt_plan inner = nullptr;
    const double* B = nullptr;
    const double* D = nullptr;
    const double* C = nullptr;
    double* Zl = nullptr;     // T^{-1} (B_1 e_1)         [(N-2) m][m]
    double* Zr = nullptr;     // T^{-1} (C_{N-2} e_{N-2}) [(N-2) m][m]
    double* U = nullptr;      // coupling columns being solved for
    double* Sinv = nullptr;   // [2m][2m]
    double* xb = nullptr;     // [2m][32] end-separator values of the last solve
    long long* status = nullptr;
    long long* status_host = nullptr;
    bool factored = false;
};

namespace {

constexpr int kThreads = 256;

inline unsigned grid_for(long long n) {
    return (unsigned)std::max<long long>(1, std::min<long long>((n + kThreads - 1) / kThreads, 4096));
}

// S = [[D_0, B_0], [C_{N-1}, D_{N-1}]] - [[C_0 Z_1], [B_{N-1} Z_{N-2}]] and its
// inverse by Gauss-Jordan elimination with partial pivoting (one CTA; the
// augmented [S | I] in shared memory, row stride 4m + 1).
__global__ void __launch_bounds__(kThreads) k_pbt_schur(long long N, int m, const double* __restrict__ B,
                                                        const double* __restrict__ D,
                                                        const double* __restrict__ C,
                                                        const double* __restrict__ Zl,
                                                        const double* __restrict__ Zr, double* __restrict__ Sinv,
                                                        long long* status) {
    extern __shared__ double sm[];
    const int n2 = 2 * m, ld = 2 * n2 + 1;
    double* a = sm;                       // [2m][ld]
    __shared__ int piv;
    __shared__ double col[64];
    const long long mm = (long long)m * m, last = N - 1, zl = (N - 3) * mm;   // Z block of the last inner row
    for (int e = threadIdx.x; e < n2 * n2; e += blockDim.x) {
        const int r = e / n2, c = e % n2;
        const int rb = r / m, rr = r % m, cb = c / m, cc = c % m;
        double v;
        if (rb == 0) {
            // row 0: D_0 (x_0), B_0 (x_{N-1}) minus C_0 times the first inner row of Z
            v = (cb == 0 ? D[rr * m + cc] : B[rr * m + cc]);
            const double* Z = (cb == 0 ? Zl : Zr);
            for (int k = 0; k < m; ++k) v = fma(-C[rr * m + k], Z[k * m + cc], v);
        } else {
            // row N-1: C_{N-1} (x_0), D_{N-1} (x_{N-1}) minus B_{N-1} times the last inner row of Z
            v = (cb == 0 ? C[last * mm + rr * m + cc] : D[last * mm + rr * m + cc]);
            const double* Z = (cb == 0 ? Zl : Zr) + zl;
            for (int k = 0; k < m; ++k) v = fma(-B[last * mm + rr * m + k], Z[k * m + cc], v);
        }
        a[r * ld + c] = v;
        a[r * ld + n2 + c] = (r == c) ? 1.0 : 0.0;
    }
    __syncthreads();
    for (int k = 0; k < n2; ++k) {
        if (threadIdx.x == 0) {
            int p = k;
            double best = fabs(a[k * ld + k]);
            for (int r = k + 1; r < n2; ++r) {
                const double t = fabs(a[r * ld + k]);
                if (t > best) {
                    best = t;
                    p = r;
                }
            }
            piv = p;
            if (!(best > 0.0) || !(best <= 1.7976931348623157e308)) {
                if (atomicCAS(reinterpret_cast<unsigned long long*>(status), 0ull,
                              (unsigned long long)(best > 0.0 ? BT_ERR_NONFINITE : BT_ERR_SINGULAR)) == 0ull) {
                    status[1] = -1;
                    status[2] = -1;
                    status[3] = k;
                }
            }
        }
        __syncthreads();
        const int p = piv;
        if (p != k)
            for (int c = threadIdx.x; c < 2 * n2; c += blockDim.x) {
                const double t = a[k * ld + c];
                a[k * ld + c] = a[p * ld + c];
                a[p * ld + c] = t;
            }
        __syncthreads();
        const double inv = 1.0 / a[k * ld + k];
        __syncthreads();
        for (int c = threadIdx.x; c < 2 * n2; c += blockDim.x) a[k * ld + c] *= inv;
        for (int r = threadIdx.x; r < n2; r += blockDim.x) col[r] = a[r * ld + k];
        __syncthreads();
        for (int e = threadIdx.x; e < n2 * 2 * n2; e += blockDim.x) {
            const int r = e / (2 * n2), c = e % (2 * n2);
            if (r != k) a[r * ld + c] = fma(-col[r], a[k * ld + c], a[r * ld + c]);
        }
        __syncthreads();
    }
    for (int e = threadIdx.x; e < n2 * n2; e += blockDim.x) Sinv[e] = a[(e / n2) * ld + n2 + e % n2];
}

// The end separators of a solve: g = [f_0 - C_0 y_1; f_{N-1} - B_{N-1} y_{N-2}],
// [x_0; x_{N-1}] = S^{-1} g into X and xb (one CTA; y = X rows 1..N-2).
__global__ void __launch_bounds__(kThreads) k_pbt_ends(long long N, int m, int nr, const double* __restrict__ B,
                                                       const double* __restrict__ C, const double* __restrict__ Sinv,
                                                       const double* __restrict__ F, double* __restrict__ X,
                                                       double* __restrict__ xb) {
    __shared__ double g[64 * 32];
    const int n2 = 2 * m;
    const long long mm = (long long)m * m, last = N - 1, row = (long long)m * nr;
    for (int e = threadIdx.x; e < n2 * nr; e += blockDim.x) {
        const int r = e / nr, c = e % nr, rr = r % m;
        double v;
        if (r < m) {
            v = F[rr * nr + c];
            for (int k = 0; k < m; ++k) v = fma(-C[rr * m + k], X[row + k * nr + c], v);
        } else {
            v = F[last * row + rr * nr + c];
            for (int k = 0; k < m; ++k) v = fma(-B[last * mm + rr * m + k], X[(last - 1) * row + k * nr + c], v);
        }
        g[e] = v;
    }
    __syncthreads();
    for (int e = threadIdx.x; e < n2 * nr; e += blockDim.x) {
        const int r = e / nr, c = e % nr;
        double v = 0.0;
        for (int k = 0; k < n2; ++k) v = fma(Sinv[r * n2 + k], g[k * nr + c], v);
        xb[e] = v;
        if (r < m) X[r * nr + c] = v;
        else X[last * row + (r - m) * nr + c] = v;
    }
}

// x_{1..N-2} -= Zl x_0 + Zr x_{N-1}.
__global__ void __launch_bounds__(kThreads) k_pbt_update(long long N, int m, int nr, const double* __restrict__ Zl,
                                                         const double* __restrict__ Zr,
                                                         const double* __restrict__ xb, double* __restrict__ X) {
    const long long n = (N - 2) * m * nr, row = (long long)m * nr;
    for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (long long)gridDim.x * blockDim.x) {
        const long long i = e / nr;   // inner unknown
        const int c = (int)(e % nr);
        double v = X[row + e];
        for (int k = 0; k < m; ++k) {
            v = fma(-Zl[i * m + k], xb[k * nr + c], v);
            v = fma(-Zr[i * m + k], xb[(m + k) * nr + c], v);
        }
        X[row + e] = v;
    }
}

// R = F - A X with the couplings taken cyclically (FP64).
__global__ void __launch_bounds__(kThreads) k_pbt_resid(long long N, int m, int nr, const double* __restrict__ B,
                                                        const double* __restrict__ D,
                                                        const double* __restrict__ C,
                                                        const double* __restrict__ F,
                                                        const double* __restrict__ X, double* __restrict__ R) {
    const long long n = N * m * nr, mm = (long long)m * m, row = (long long)m * nr;
    for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (long long)gridDim.x * blockDim.x) {
        const long long j = e / row;
        const int r = (int)((e / nr) % m), c = (int)(e % nr);
        const long long jl = (j == 0) ? N - 1 : j - 1, jr = (j == N - 1) ? 0 : j + 1;
        double v = F[e];
        for (int k = 0; k < m; ++k) {
            v = fma(-B[j * mm + r * m + k], X[jl * row + k * nr + c], v);
            v = fma(-D[j * mm + r * m + k], X[j * row + k * nr + c], v);
            v = fma(-C[j * mm + r * m + k], X[jr * row + k * nr + c], v);
        }
        R[e] = v;
    }
}

bt_status from_cuda(cudaError_t e) {
    if (e == cudaSuccess) return BT_OK;
    return e == cudaErrorMemoryAllocation ? BT_ERR_NOMEM : BT_ERR_CUDA;
}

size_t schur_smem(int m) { return sizeof(double) * (size_t)(2 * m) * (4 * m + 1); }

}  // namespace

extern "C" {

bt_status pbt_plan_create(pbt_plan* out, int64_t N, int m, int nrhs_max, int64_t p, void* stream) {
    if (!out) return BT_ERR_INVALID;
    *out = nullptr;
    if (N < 4 || m < 1 || m > 32 || nrhs_max < 1 || nrhs_max > 32 || p < 0) return BT_ERR_INVALID;
    pbt_plan_s* P = new (std::nothrow) pbt_plan_s();
    if (!P) return BT_ERR_NOMEM;
    P->N = N;
    P->m = m;
    P->nrhs_max = nrhs_max;
    P->stream = (cudaStream_t)stream;
    bt_status st = bt_plan_create(&P->inner, N - 2, m, std::max(nrhs_max, m), BT_FP64, p, stream);
    if (st != BT_OK) {
        delete P;
        return st;
    }
    const size_t zbytes = sizeof(double) * (size_t)(N - 2) * m * m;
    cudaError_t e = cudaMalloc((void**)&P->Zl, zbytes);
    if (e == cudaSuccess) e = cudaMalloc((void**)&P->Zr, zbytes);
    if (e == cudaSuccess) e = cudaMalloc((void**)&P->U, zbytes);
    if (e == cudaSuccess) e = cudaMalloc((void**)&P->Sinv, sizeof(double) * 4 * m * m);
    if (e == cudaSuccess) e = cudaMalloc((void**)&P->xb, sizeof(double) * 2 * m * 32);
    if (e == cudaSuccess) e = cudaMalloc((void**)&P->status, 4 * sizeof(long long));
    if (e == cudaSuccess) e = cudaMallocHost((void**)&P->status_host, 4 * sizeof(long long));
    if (e == cudaSuccess) e = cudaMemsetAsync(P->status, 0, 4 * sizeof(long long), P->stream);
    if (e == cudaSuccess && schur_smem(m) > 48 * 1024)
        e = cudaFuncSetAttribute(k_pbt_schur, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)schur_smem(m));
    if (e != cudaSuccess) {
        pbt_plan_destroy(P);
        cudaGetLastError();
        return from_cuda(e);
    }
    *out = P;
    return BT_OK;
}

bt_status pbt_factor(pbt_plan P, const double* B, const double* D, const double* C) {
    if (!P || !B || !D || !C) return BT_ERR_INVALID;
    const long long N = P->N, mm = (long long)P->m * P->m, inner = N - 2;
    P->B = B;
    P->D = D;
    P->C = C;
    P->factored = false;
    cudaError_t e = cudaMemsetAsync(P->status, 0, 4 * sizeof(long long), P->stream);
    if (e != cudaSuccess) return from_cuda(e);
    bt_status st = bt_factor(P->inner, B + mm, D + mm, C + mm);
    if (st != BT_OK) return st;
    // Z columns: T^{-1} of the first inner row's coupling B_1 to x_0, and of the
    // last inner row's coupling C_{N-2} to x_{N-1}
    const size_t zbytes = sizeof(double) * (size_t)inner * mm;
    e = cudaMemsetAsync(P->U, 0, zbytes, P->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(P->U, B + mm, sizeof(double) * mm, cudaMemcpyDeviceToDevice, P->stream);
    if (e != cudaSuccess) return from_cuda(e);
    st = bt_solve(P->inner, P->U, P->Zl, P->m);
    if (st != BT_OK) return st;
    e = cudaMemsetAsync(P->U, 0, zbytes, P->stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(P->U + (inner - 1) * mm, C + (N - 2) * mm, sizeof(double) * mm, cudaMemcpyDeviceToDevice,
                            P->stream);
    if (e != cudaSuccess) return from_cuda(e);
    st = bt_solve(P->inner, P->U, P->Zr, P->m);
    if (st != BT_OK) return st;
    k_pbt_schur<<<1, kThreads, schur_smem(P->m), P->stream>>>(N, P->m, B, D, C, P->Zl, P->Zr, P->Sinv, P->status);
    e = cudaGetLastError();
    if (e != cudaSuccess) return from_cuda(e);
    P->factored = true;
    return BT_OK;
}

bt_status pbt_solve(pbt_plan P, const double* F, double* X, int nrhs) {
    if (!P || !F || !X || nrhs < 1 || nrhs > P->nrhs_max || !P->factored) return BT_ERR_INVALID;
    const long long row = (long long)P->m * nrhs;
    bt_status st = bt_solve(P->inner, F + row, X + row, nrhs);
    if (st != BT_OK) return st;
    k_pbt_ends<<<1, kThreads, 0, P->stream>>>(P->N, P->m, nrhs, P->B, P->C, P->Sinv, F, X, P->xb);
    k_pbt_update<<<grid_for((P->N - 2) * row), kThreads, 0, P->stream>>>(P->N, P->m, nrhs, P->Zl, P->Zr, P->xb, X);
    return from_cuda(cudaGetLastError());
}

bt_status pbt_residual(pbt_plan P, const double* F, const double* X, double* R, int nrhs) {
    if (!P || !F || !X || !R || nrhs < 1 || nrhs > P->nrhs_max || !P->B) return BT_ERR_INVALID;
    k_pbt_resid<<<grid_for(P->N * P->m * nrhs), kThreads, 0, P->stream>>>(P->N, P->m, nrhs, P->B, P->D, P->C, F, X,
                                                                          R);
    return from_cuda(cudaGetLastError());
}

bt_status pbt_sync(pbt_plan P) {
    if (!P) return BT_ERR_INVALID;
    bt_status st = bt_sync(P->inner);
    cudaError_t e = cudaMemcpyAsync(P->status_host, P->status, 4 * sizeof(long long), cudaMemcpyDeviceToHost,
                                    P->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(P->stream);
    if (e != cudaSuccess) return from_cuda(e);
    if (st != BT_OK) return st;
    return (bt_status)P->status_host[0];
}

void pbt_plan_destroy(pbt_plan P) {
    if (!P) return;
    if (P->inner) bt_plan_destroy(P->inner);
    cudaFree(P->Zl);
    cudaFree(P->Zr);
    cudaFree(P->U);
    cudaFree(P->Sinv);
    cudaFree(P->xb);
    cudaFree(P->status);
    if (P->status_host) cudaFreeHost(P->status_host);
    delete P;
}

}  // extern "C"
