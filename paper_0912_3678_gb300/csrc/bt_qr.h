// Partitions factored by QR (Sec. 2, the variant with N^(i) = Q^(i) and
// S^(i) = R^(i)): every partition's local block A^(i) is reduced to R^(i) by
// block Householder steps, one CTA per partition in FP64; the reduced matrix
// T_p (Eq. (redmatr)) is assembled from the spikes and solved by the pivoted
// direct solver.
//
// With the partition's local rows s..e-1 and its separators s-1 (left, when
// i > 0) and e (right, when i < p-1), Eq. (parblock) with N = Q, S = R gives
//   z = Q^T b_0              left separator column (fill-in, every row),
//   y = Q^T c_1              right separator column (rows e-2, e-1 only),
//   w^T = c_0^T R^{-1}       left separator row (fill-in, every row),
//   v^T = b_1^T R^{-1}       right separator row (block e-1 only),
// and the partition's share of T_p: -w^T z on the left separator's diagonal,
// -w^T y coupling left to right, -v^T z coupling right to left and
// a_e - v^T y on the right separator's diagonal.
//
// Storage, per local block row j (block order m, row-major m x m blocks):
//   Qt[j]  [2m][2m]  Q_j^T of the step at row j: the 2m x 2m orthogonal
//                    factor that reduces [D~_j; B_{j+1}] to [R_jj; 0]; the
//                    last local row of a partition reduces D~_j alone and
//                    keeps Q_j^T in the leading m x m corner;
//   R[j]   [3][m][m] R_jj (upper triangular), R_{j,j+1}, R_{j,j+2}, where a
//                    block column e is the right separator (y) and e + 1 is
//                    zero;
//   Z[j]   [m][m]    z_j;
//   W[j]   [m][m]    w_j^T;
// per partition: Vb [m][m] v^T_{e-1}, Ta [m][m] -w^T z, Tf [m][nr] w^T of the
// forward-substituted right-hand side.
#pragma once
#include <cuda_runtime.h>

namespace bt {

struct QrArgs {
    long long N, p, base, extra;   // level-0 geometry (uniform split, as part_bounds)
    int m, nr;
    const double* B;
    const double* D;
    const double* C;
    double* Qt;
    double* R;
    double* Z;
    double* W;
    double* Vb;
    double* Ta;
    double* Tf;
    double* Bn;          // reduced matrix [p-1][m][m]
    double* Dn;
    double* Cn;
    const double* F;     // [N][m][nr]
    double* X;           // [N][m][nr]: u_j = Q^T f between the two solve passes
    double* Fn;          // reduced right-hand side [p-1][m][nr]
    const double* Xn;    // reduced solution [p-1][m][nr]
    long long* status;
};

// Factorization: one launch of the local QR factorizations plus one that adds
// the left partitions' shares into the reduced diagonal (2 kernels).
cudaError_t launch_qr_factor(const QrArgs& a, cudaStream_t s);
// Forward pass u = Q^T f with the separators' right-hand sides (2 kernels).
cudaError_t launch_qr_solve_fwd(const QrArgs& a, cudaStream_t s);
// Back substitution with R and the separator values (1 kernel).
cudaError_t launch_qr_solve_bwd(const QrArgs& a, cudaStream_t s);
// Dynamic shared memory limits of the three kernels for block order m.
cudaError_t qr_prepare(int m);

}  // namespace bt
