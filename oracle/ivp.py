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
