// Single-launch solve of the reduced system by block cyclic reduction for the
// refined paths (bt_rsolve.cu).
#pragma once
#include <cuda_runtime.h>

namespace bt {

constexpr int kRsMaxLevels = 28;

// FP32 copies of a cyclic-reduction factorization (levels q = 0..nlev-1 with
// K[q] active block rows, the last one K == 1) and FP32 level vectors.
struct RsolveArgs {
    int nlev, m, nr;
    long long K[kRsMaxLevels];
    const float* al[kRsMaxLevels];    // [(K+1)/2][m][m]  multipliers of the kept rows (left)
    const float* ga[kRsMaxLevels];    // [(K+1)/2][m][m]  (right)
    const float* Dinv[kRsMaxLevels];  // [K/2][m][m] inverses of the odd rows (K == 1: [1])
    const float* B[kRsMaxLevels];     // [K][m][m] level matrix (the odd rows are used)
    const float* C[kRsMaxLevels];
    float* f[kRsMaxLevels];           // [K][m][nr] right-hand side of the level
    float* x[kRsMaxLevels];           // [K][m][nr] solution of the level
    const double* F0;                 // level-0 right-hand side (FP64)
    double* X0;                       // level-0 solution (FP64)
    // Set by launch_rsolve_f32: levels [0, big) run on the whole cluster with
    // `chunk` floats of shared memory for their chunks; levels [big, nlev) run
    // on CTA 0 from shared memory, level q's blocks and vector at offset
    // soff[q] (floats) past the chunk area.
    int big, chunk;
    int soff[kRsMaxLevels + 1];
};

// Conversion of FP64 arrays to FP32 (rounded to nearest): up to kCvtSegs
// segments in one launch.
constexpr int kCvtSegs = 5 * kRsMaxLevels;
struct CvtArgs {
    int nseg;
    const double* src[kCvtSegs];
    float* dst[kCvtSegs];
    long long n[kCvtSegs];
};

// One-launch FP32 cyclic-reduction factorization of the reduced system (the
// refined paths, block orders 8 and 16): level q has K[q] rows; its matrix is
// the FP64 B0, D0, C0 for q = 0 and the FP32 B[q], D[q], C[q] above; it
// writes al[q], ga[q] ((K+1)/2 blocks), Dinv[q] (K/2 blocks, 1 when K == 1)
// and the next level's matrix B[q+1], D[q+1], C[q+1].
struct RfactorArgs {
    int nlev, m, level0;   // level0: the plan level number of q = 0 (status reports)
    long long K[kRsMaxLevels];
    const double* B0;
    const double* D0;
    const double* C0;
    float* B[kRsMaxLevels];
    float* D[kRsMaxLevels];
    float* C[kRsMaxLevels];
    float* al[kRsMaxLevels];
    float* ga[kRsMaxLevels];
    float* Dinv[kRsMaxLevels];
    float* B0f;            // FP32 copies of B0 and C0 for the solves ([K[0]][m][m]; the odd
    float* C0f;            // rows, the only ones the solves read, are written)
    long long* status;
};

cudaError_t launch_cvt_f32(const CvtArgs& a, cudaStream_t s);
// m in {8, 16}
cudaError_t launch_rfactor_f32(const RfactorArgs& a, cudaStream_t s);
// m in {8, 16, 32}
cudaError_t launch_rsolve_f32(const RsolveArgs& a, cudaStream_t s);

}  // namespace bt
