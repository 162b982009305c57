// Launchers for the FP64 residual, refinement and small direct-solve kernels.
#pragma once
#include <cuda_runtime.h>

namespace bt {
// Maxima are merged with integer atomicMax into kMaxSlots slots of 3 words
// (slot = block index mod kMaxSlots, spreading the atomics); the caller zeroes
// them first and takes the maximum over the slots.
constexpr int kMaxSlots = 32;
// maxout (may be null): [kMaxSlots][3] bit patterns of max |r|, max |x|, max |f|
cudaError_t launch_resid_btri(long long N, int m, int nr, const double* B, const double* D, const double* C,
                              const double* X, const double* F, double* R, cudaStream_t s,
                              unsigned long long* maxout = nullptr);
cudaError_t launch_resid_babd(long long N, int m, int nr, const double* S, const double* Rm, const double* B0,
                              const double* B1, const double* Y, const double* F, double* Rout, cudaStream_t s,
                              unsigned long long* maxout = nullptr);
// out: [kMaxSlots][3], ||A||_inf (bit pattern) in word 0 of each slot
cudaError_t launch_norm_inf(int kind, long long N, int m, const double* A0, const double* A1, const double* A2,
                            const double* B0, const double* B1, unsigned long long* out, cudaStream_t s);
int ir_update_blocks(long long n);
// out[0..1] = sums over the n pairs partial[2i], partial[2i+1] (one CTA, fixed order)
cudaError_t launch_reduce_pairs(int n, const double* partial, double* out, cudaStream_t s);
cudaError_t launch_ir_update(long long n, double* X, const double* Dc, double* partial, double* out,
                             cudaStream_t s);
size_t babd_direct_smem(int m, int nr);
// Small block tridiagonal system (K block rows) by banded GEPP in one CTA;
// keep: [K][m][3m+nr] doubles of workspace.
size_t btri_direct_smem(int m, int nr);
cudaError_t launch_btri_direct(int K, int m, int nr, const double* B, const double* D, const double* C,
                               const double* F, double* X, double* keep, long long* status, int level,
                               cudaStream_t s);
cudaError_t launch_babd_direct(int Np, int m, int nr, const double* S, const double* R, const double* B0,
                               const double* B1, const double* F, double* X, double* keep, long long* status,
                               int level, cudaStream_t s);
}  // namespace bt

namespace bt {
cudaError_t launch_pad_blocks(long long N, int m, int M, const double* in, double* out, int identity_tail,
                              cudaStream_t s);
cudaError_t launch_pad_rhs(long long rows, int m, int M, int nr, const double* in, double* out, cudaStream_t s);
cudaError_t launch_unpad_rhs(long long rows, int m, int M, int nr, const double* in, double* out, cudaStream_t s);
cudaError_t launch_band_to_blocks(long long n, int s, int r, const double* band, long long N, int m, double* B,
                                  double* D, double* C, cudaStream_t stream);
}  // namespace bt

namespace bt {
// Refinement residuals in double-float arithmetic on the FP32 pipe (compensated
// dot products, bt_resid_df.cu): entries accurate to a few units of 2^-48 of
// sum |a||x| + |f|, returned rounded to FP32 precision in FP64 storage; same
// arguments and maxima slots as launch_resid_btri / launch_resid_babd.
size_t resid_df_smem(int kind, int m, int nr);
cudaError_t launch_resid_btri_df(long long N, int m, int nr, const double* B, const double* D, const double* C,
                                 const double* X, const double* F, double* R, cudaStream_t s,
                                 unsigned long long* maxout = nullptr);
// The same residual for order 16 with the matrix kept as the warp-per-partition
// factorization's split copy (B, D, C as negated FP32 (hi, lo) parts by column
// pairs, the bytes of float2 [3][N][16][16]).
// The same residual with the products on the tensor cores (block tridiagonal,
// m = 16, nr <= 8; cudaErrorInvalidValue otherwise): Ozaki splitting into
// 8-bit digit planes, BF16 mma.sync with FP32 accumulation, double-float
// combination; the result rounded to FP32 precision (bt_resid_df.cu).
cudaError_t launch_resid_btri_oz(long long N, int m, int nr, const double* B, const double* D, const double* C,
                                 const double* X, const double* F, double* R, cudaStream_t s,
                                 unsigned long long* maxout);
cudaError_t launch_resid_btri_dfs(long long N, int m, int nr, const float2* As, const double* X, const double* F,
                                  double* R, cudaStream_t s, unsigned long long* maxout = nullptr);
cudaError_t launch_resid_babd_df(long long N, int m, int nr, const double* S, const double* Rm, const double* B0,
                                 const double* B1, const double* Y, const double* F, double* Rout, cudaStream_t s,
                                 unsigned long long* maxout = nullptr);
}  // namespace bt
