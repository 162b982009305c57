/* Parallel-in-time solution of linear ODE initial-value problems (Secs. 3 and
 * 4 of Amodio & Brugnano, "Parallel Factorizations in Numerical Analysis"):
 * the Parareal iteration as the iterative solution of the reduced system
 * (redsys) by the splitting F = (F - G) + G with a cheap coarse propagator G.
 *
 * Problem: y' = L y + g(t), y(0) = y0, t in [0, T], with L tridiagonal of
 * order n (dl, d, du: dl[0] and du[n-1] unused) -- the method of lines for a
 * 1-D parabolic problem is the case the paper has in mind -- and affine
 * forcing g(t) = g0 + t g1.  Coarse mesh tau_i = i T / p, i = 0..p (Eq.
 * (coarse)).
 *
 * Propagators: F_i = nfine steps of the trapezoidal rule on [tau_i, tau_{i+1}]
 * (each step one tridiagonal solve with I - h/2 L, all p intervals advanced
 * together as p right-hand sides of one solve); G_i = ncoarse steps of
 * backward Euler (one tridiagonal solve with I - h_c L per step, sequential
 * over the intervals).  Both tridiagonal solves are the partition-method
 * plans of bt.h (m = 1).
 *
 * Iteration (Eq. (parareal1)): U_0 = y0, U_{i+1}^(0) = G_i U_i^(0); then
 *   U_{i+1}^(k+1) = G_i U_i^(k+1) + F_i U_i^(k) - G_i U_i^(k),
 * stopped when max_i ||U_i^(k+1) - U_i^(k)||_inf <= tol max_i ||U_i^(k+1)||_inf
 * or after kmax iterations (kmax <= p: after p iterations U equals the
 * sequential fine solution).
 *
 * Arguments (device pointers unless stated): dl, d, du, g0, y0 [n]; g1 [n]
 * or NULL; U [p+1][n] output, U[i] ~ y(tau_i); hist NULL or
 * [(kmax+1)][p+1][n] output of every iterate; iters_out (host, may be NULL):
 * iterations done; 1 <= p <= 32, nfine >= 1, ncoarse >= 1, 0 <= kmax <= p,
 * T > 0.  Allocates its workspace (cudaMalloc) and synchronises the stream.
 * Errors: BT_ERR_INVALID for bad arguments, BT_ERR_SINGULAR / BT_ERR_NONFINITE
 * from the tridiagonal solves, BT_ERR_NOT_CONVERGED when kmax iterations end
 * above tol (U then holds the last iterate). */
#pragma once
#include <stdint.h>

#include "bt.h"

#ifdef __cplusplus
extern "C" {
#endif

bt_status ivp_parareal(int64_t n, const double* dl, const double* d, const double* du, const double* g0,
                       const double* g1, const double* y0, double T, int p, int nfine, int ncoarse, int kmax,
                       double tol, double* U, double* hist, int* iters_out, void* stream);

/* Parallel IVP solver with a block Boundary Value Method as the local method
 * (Sec. 3, Eqs. (M_iy_i), (My), (D), (redsys), (pups)).
 *
 * Problem: y' = L y + g(t), y(0) = y0, t in [0, T], L a constant m x m matrix.
 * Coarse mesh of p equal intervals (Eq. (coarse)), N steps of h = T / (p N) in
 * each (Eq. (hi)).  Local method: the order-3 generalized Adams BVM with
 * k = 2, y_n - y_{n-1} = h (5/12 f_{n-1} + 2/3 f_n - 1/12 f_{n+1}) for
 * n = 1..N-1 (coefficients from the order conditions), and the trapezoidal
 * rule y_N - y_{N-1} = h/2 (f_{N-1} + f_N) as final formula, so that every
 * M_i is block tridiagonal (and, with constant L, the same matrix M).
 * Steps: (D) M z_i = g_i for every interval and the propagator
 * w = M^{-1} v, one partition-method factorization of M (bt_plan, FP64) and
 * its solves; (redsys) y_{0,1} = y0, y_{0,i+1} = z_{N,i} + w_N y_{0,i};
 * (pups) y_i = z_i + w y_{0,i}.
 *
 * Arguments (device pointers): L [m][m] row-major; y0 [m]; G [p N + 1][m]
 * with G[k] = g(k h) on the fine grid; Y [p N + 1][m] output, Y[k] ~ y(k h)
 * (Y[0] = y0).  1 <= m <= 32, p >= 1, N >= 1, T > 0.  Allocates its workspace
 * (cudaMalloc), runs on `stream` and synchronises it.  Errors:
 * BT_ERR_INVALID for bad arguments, BT_ERR_NOMEM, BT_ERR_SINGULAR /
 * BT_ERR_NONFINITE from the factorization of M. */
bt_status ivp_bvm(int m, int64_t p, int64_t N, double T, const double* L, const double* y0, const double* G,
                  double* Y, void* stream);

#ifdef __cplusplus
}
#endif
