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

cudaError_t launch_cvt_f32(const CvtArgs& a, cudaStream_t s);
// m in {8, 16, 32}
cudaError_t launch_rsolve_f32(const RsolveArgs& a, cudaStream_t s);

}  // namespace bt
