"""Oracle for the parallel IVP solver and Parareal (Secs. 3 and 4 of the paper).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``): plain sequential FP64
propagators and the Parareal iteration written out step by step, for the
linear ODE-IVP

    y' = L y + g(t),  y(0) = y0,  t in [0, T],  L tridiagonal (order n),
    g(t) = g0 + t g1,

with a coarse mesh of p equal intervals tau_i = i T / p (Eq. (coarse)).

* ``fine``    the fine propagator F_i of one interval: nfine steps of the
              trapezoidal rule, (I - h/2 L) y_{k+1} = (I + h/2 L) y_k
              + h/2 (g(t_k) + g(t_{k+1})), each step one tridiagonal solve by
              the oracle's Thomas algorithm;
* ``coarse``  the coarse propagator G_i: ncoarse backward Euler steps,
              (I - h_c L) y_{k+1} = y_k + h_c g(t_{k+1});
* ``parareal`` the iteration of Eq. (parareal1),
              y_{0,1} = y0,
              y_{0,i+1}^{(k+1)} = G_i y_{0,i}^{(k+1)} + (F_i - G_i) y_{0,i}^{(k)},
              started from the sequential coarse sweep (k = 0); it solves the
              reduced system (redsys) iteratively and returns every iterate.
* ``laplacian`` / ``eig_*``: the 1-D Dirichlet heat operator and its closed
              form eigenpairs, for the pins.
* ``gam3_coefficients``, ``bvm_blocks``, ``bvm_rhs``, ``bvm_sequential``:
              the parallel IVP solver of Sec. 3 with a block Boundary Value
              Method as the local solver (general block tridiagonal M_i):
              the discrete problem (My) solved by its sequential recursion.
"""
from __future__ import annotations

import numpy as np

from . import tri_solve


def laplacian(n: int, nu: float = 1.0):
    """L = nu/dx^2 tridiag(1, -2, 1) on n interior points of [0, 1] (dx = 1/(n+1));
    returns (dl, d, du) with dl[0] = du[n-1] = 0."""
    dx = 1.0 / (n + 1)
    c = nu / (dx * dx)
    dl = np.full(n, c)
    du = np.full(n, c)
    d = np.full(n, -2.0 * c)
    dl[0] = 0.0
    du[-1] = 0.0
    return dl, d, du


def eig_laplacian(n: int, nu: float = 1.0):
    """Eigenvalues lambda_k = -4 nu/dx^2 sin^2(k pi / (2(n+1))) and the
    orthonormal eigenvectors v_k(j) = sqrt(2/(n+1)) sin(j k pi/(n+1)),
    k, j = 1..n (columns of V)."""
    dx = 1.0 / (n + 1)
    k = np.arange(1, n + 1)
    lam = -4.0 * nu / (dx * dx) * np.sin(k * np.pi / (2 * (n + 1))) ** 2
    j = np.arange(1, n + 1)
    V = np.sqrt(2.0 / (n + 1)) * np.sin(np.outer(j, k) * np.pi / (n + 1))
    return lam, V


def _matvec(dl, d, du, y):
    """L y for the tridiagonal L."""
    out = d * y
    out[1:] += dl[1:] * y[:-1]
    out[:-1] += du[:-1] * y[1:]
    return out


def fine(dl, d, du, y, g0, g1, t0: float, h: float, nsteps: int):
    """nsteps trapezoidal steps of size h from y at time t0."""
    y = np.array(y, dtype=np.float64)
    g1 = np.zeros_like(y) if g1 is None else g1
    A = (-0.5 * h * dl, 1.0 - 0.5 * h * d, -0.5 * h * du)
    for k in range(nsteps):
        tk = t0 + k * h
        rhs = y + 0.5 * h * _matvec(dl, d, du, y) + 0.5 * h * (2.0 * g0 + g1 * (2.0 * tk + h))
        y = tri_solve(A[0], A[1], A[2], rhs)
    return y


def coarse(dl, d, du, y, g0, g1, t0: float, H: float, nsteps: int):
    """nsteps backward Euler steps covering H from y at time t0."""
    y = np.array(y, dtype=np.float64)
    g1 = np.zeros_like(y) if g1 is None else g1
    hc = H / nsteps
    A = (-hc * dl, 1.0 - hc * d, -hc * du)
    for k in range(nsteps):
        t1 = t0 + (k + 1) * hc
        y = tri_solve(A[0], A[1], A[2], y + hc * (g0 + g1 * t1))
    return y


def sequential_fine(dl, d, du, y0, g0, g1, T: float, p: int, nfine: int):
    """The fine solution at the coarse points tau_0..tau_p, interval after
    interval (the sequential recursion of the reduced system, Eq. (recur))."""
    H = T / p
    out = [np.array(y0, dtype=np.float64)]
    for i in range(p):
        out.append(fine(dl, d, du, out[-1], g0, g1, i * H, H / nfine, nfine))
    return np.array(out)


def parareal(dl, d, du, y0, g0, g1, T: float, p: int, nfine: int, ncoarse: int, kmax: int):
    """All Parareal iterates U[k][i] ~ y(tau_i), k = 0..kmax (Eq. (parareal1))."""
    H = T / p
    Fi = lambda i, y: fine(dl, d, du, y, g0, g1, i * H, H / nfine, nfine)
    Gi = lambda i, y: coarse(dl, d, du, y, g0, g1, i * H, H, ncoarse)
    U = [np.array(y0, dtype=np.float64)]
    for i in range(p):                        # k = 0: the sequential coarse sweep
        U.append(Gi(i, U[i]))
    iters = [np.array(U)]
    for k in range(kmax):
        Uk = iters[-1]
        Fv = [Fi(i, Uk[i]) for i in range(p)]         # parallel over i
        Gv = [Gi(i, Uk[i]) for i in range(p)]
        Un = [np.array(y0, dtype=np.float64)]
        for i in range(p):                            # sequential correction sweep
            Un.append(Gi(i, Un[i]) + Fv[i] - Gv[i])
        iters.append(np.array(Un))
    return np.array(iters)


# --------------------------------------------------------------------------
# Parallel IVP solver with a block Boundary Value Method (Sec. 3, Eqs.
# (M_iy_i), (My)) for y' = L y + g(t), L a constant m x m matrix, y(0) = y0.
# Coarse mesh of p equal intervals, N steps of h = T / (p N) in each.
#
# Method: the generalized Adams BVM with k = 2 steps (nu = 1 initial value)
# as main formula,
#     y_n - y_{n-1} = h (b0 f_{n-1} + b1 f_n + b2 f_{n+1}),  n = 1..N-1,
# its coefficients fixed by exactness on polynomials of degree <= 3 (order
# 3), and the trapezoidal rule as the final additional formula
#     y_N - y_{N-1} = h/2 (f_{N-1} + f_N),
# which keeps M_i block tridiagonal.  With f = L y + g, block row n of M_i is
#     B_n y_{n-1} + D_n y_n + C_n y_{n+1} = r_n,
# and the row n = 1 term B_1 y_0 is moved to the right: v_i = -B_1.
# --------------------------------------------------------------------------
def gam3_coefficients():
    """(b0, b1, b2) as exact fractions: exactness of the main formula on
    y = t^q, q = 1..3, with the nodes t_{n-1} = 0, t_n = 1, t_{n+1} = 2 (h = 1),
    i.e. y(1) - y(0) = 1 = sum_j b_j q j^(q-1) (with 0^0 = 1), solved by
    Gauss-Jordan elimination in rational arithmetic."""
    from fractions import Fraction
    rows = [[Fraction(q) * Fraction(j) ** (q - 1) for j in (0, 1, 2)] + [Fraction(1)] for q in (1, 2, 3)]
    for c in range(3):
        piv = next(r for r in range(c, 3) if rows[r][c] != 0)
        rows[c], rows[piv] = rows[piv], rows[c]
        pv = rows[c][c]
        rows[c] = [v / pv for v in rows[c]]
        for r in range(3):
            if r != c and rows[r][c] != 0:
                f = rows[r][c]
                rows[r] = [a - f * b for a, b in zip(rows[r], rows[c])]
    return tuple(rows[c][3] for c in range(3))


def bvm_blocks(L, h: float, N: int):
    """Block rows of the local matrix M_i (identical for every interval):
    B, D, C of shape [N][m][m] (B[0] and C[N-1] unused) and the coupling of
    row 1 to the interval's initial value, v = -B_1, shape [m][m]."""
    L = np.asarray(L, dtype=np.float64)
    m = L.shape[0]
    b0, b1, b2 = (float(c) for c in gam3_coefficients())
    I = np.eye(m)
    B = np.zeros((N, m, m))
    D = np.zeros((N, m, m))
    C = np.zeros((N, m, m))
    for n in range(N):                       # row n + 1 of the interval
        if n < N - 1:                        # main formula
            B[n] = -(I + h * b0 * L)
            D[n] = I - h * b1 * L
            C[n] = -h * b2 * L
        else:                                # final formula (trapezoidal rule)
            B[n] = -(I + 0.5 * h * L)
            D[n] = I - 0.5 * h * L
    return B, D, C, -B[0].copy()


def bvm_rhs(Gi, h: float, N: int):
    """Right-hand sides r_n (n = 1..N) of one interval from the samples
    Gi[k] = g(tau_{i-1} + k h), k = 0..N; shape [N][m]."""
    b0, b1, b2 = (float(c) for c in gam3_coefficients())
    Gi = np.asarray(Gi, dtype=np.float64)
    r = np.zeros((N, Gi.shape[1]))
    for n in range(1, N + 1):
        if n < N:
            r[n - 1] = h * (b0 * Gi[n - 1] + b1 * Gi[n] + b2 * Gi[n + 1])
        else:
            r[n - 1] = 0.5 * h * (Gi[n - 1] + Gi[n])
    return r


def bvm_sequential(L, y0, G, T: float, p: int, N: int):
    """The discrete solution of (My) by its sequential recursion,
    y_{N0} = y0,  M_i y_i = g_i + v_i y_{N,i-1},  i = 1..p,
    each M_i solved by the oracle's block Thomas algorithm.  G holds g at
    the p N + 1 fine grid points; returns Y with Y[k] ~ y(k h)."""
    from . import btri_solve
    h = T / (p * N)
    B, D, C, v = bvm_blocks(L, h, N)
    G = np.asarray(G, dtype=np.float64)
    m = B.shape[1]
    Y = np.zeros((p * N + 1, m))
    Y[0] = np.asarray(y0, dtype=np.float64)
    for i in range(p):
        r = bvm_rhs(G[i * N:(i + 1) * N + 1], h, N)
        r[0] += v @ Y[i * N]
        y = btri_solve(B, D, C, r.reshape(N * m, 1)).reshape(N, m)
        Y[i * N + 1:(i + 1) * N + 1] = y
    return Y
