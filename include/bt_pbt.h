/* Block tridiagonal matrices with corner blocks (Sec. 2, Eqs. (parpart1),
 * (redmatr1) with the c couplings kept): for j = 0..N-1,
 *   B_j x_{j-1} + D_j x_j + C_j x_{j+1} = f_j,
 * indices taken cyclically, so B_0 couples row 0 to x_{N-1} (the right-upper
 * corner block b of Eq. (parpart1)) and C_{N-1} couples row N-1 to x_0 (the
 * left-lower corner; zero for the one-corner form of the paper, nonzero for a
 * periodic block tridiagonal matrix).  A plain block tridiagonal plan never
 * reads B_0 and C_{N-1}; these plans do.
 *
 * Partitioning: block rows 0 and N-1 are separators, the end rows a^(0) and
 * a^(p) of Eq. (parpart1); rows 1..N-2 are partitioned by an inner partition
 * method plan (bt.h) with its own separators.  The reduced system of
 * Eq. (redmatr1) -- block tridiagonal with the corner blocks -- is solved by
 * eliminating the inner separators first (the inner plan) and then the two
 * end separators: with T the block tridiagonal matrix of rows 1..N-2, the
 * couplings U = [B_1 e_1, C_{N-2} e_{N-2}] of its first and last rows to
 * x_0 and x_{N-1}, and Z = T^{-1} U (2m columns, formed at factorization time),
 *   S = [[D_0, B_0], [C_{N-1}, D_{N-1}]] - [[C_0 Z_1], [B_{N-1} Z_{N-2}]]
 * is the 2m x 2m Schur complement onto the end separators (inverted by
 * Gauss-Jordan elimination with partial pivoting); a solve is
 *   y = T^{-1} f_{1..N-2},  [x_0; x_{N-1}] = S^{-1} ([f_0; f_{N-1}] -
 *   [C_0 y_1; B_{N-1} y_{N-2}]),  x_{1..N-2} = y - Z [x_0; x_{N-1}].
 *
 * Arguments: device arrays, row-major FP64, B, D, C [N][m][m] (B_0 and
 * C_{N-1} are the corner blocks), F, X [N m][nrhs]; 4 <= N, 1 <= m <= 32,
 * 1 <= nrhs <= nrhs_max <= 32, FP64 only.  The plan keeps the matrices by
 * reference (like bt_factor) and holds Z (2 N m^2 doubles).  Calls are
 * asynchronous on the plan's stream; pbt_sync waits and returns the status.
 * Errors: BT_ERR_INVALID for bad arguments, BT_ERR_NOMEM, BT_ERR_SINGULAR /
 * BT_ERR_NONFINITE from the inner factorization or from S. */
#pragma once
#include <stdint.h>

#include "bt.h"

#ifdef __cplusplus
extern "C" {
#endif

typedef struct pbt_plan_s* pbt_plan;

/* p: partitions of the inner plan (0: its default). */
bt_status pbt_plan_create(pbt_plan* plan, int64_t N, int m, int nrhs_max, int64_t p, void* stream);
/* Factor the inner block tridiagonal part, form Z and invert S. */
bt_status pbt_factor(pbt_plan plan, const double* B, const double* D, const double* C);
/* X = A^{-1} F (F and X may not overlap). */
bt_status pbt_solve(pbt_plan plan, const double* F, double* X, int nrhs);
/* R = F - A X in FP64, with the corner couplings. */
bt_status pbt_residual(pbt_plan plan, const double* F, const double* X, double* R, int nrhs);
bt_status pbt_sync(pbt_plan plan);
void pbt_plan_destroy(pbt_plan plan);

#ifdef __cplusplus
}
#endif
