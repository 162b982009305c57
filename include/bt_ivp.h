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

#ifdef __cplusplus
}
#endif
