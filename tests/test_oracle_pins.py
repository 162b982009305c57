"""Pins of the oracle to facts fixed by mathematics, not by the oracle itself:
closed forms, exact rational arithmetic, brute-force dense LAPACK solves,
special cases that reduce to other algorithms, manufactured solutions and the
convergence order of the trapezoidal rule."""
from fractions import Fraction

import numpy as np
import pytest

import gen
import oracle


def _gepp_fraction(A, b):
    """Exact Gaussian elimination over the rationals (brute force, tiny n)."""
    n = len(A)
    M = [[Fraction(int(A[i][j])) for j in range(n)] + [Fraction(int(b[i]))] for i in range(n)]
    for k in range(n):
        p = next(i for i in range(k, n) if M[i][k] != 0)
        M[k], M[p] = M[p], M[k]
        for i in range(k + 1, n):
            f = M[i][k] / M[k][k]
            for j in range(k, n + 1):
                M[i][j] -= f * M[k][j]
    x = [Fraction(0)] * n
    for i in range(n - 1, -1, -1):
        s = M[i][n] - sum(M[i][j] * x[j] for j in range(i + 1, n))
        x[i] = s / M[i][i]
    return x


# ------------------------------------------------------------ dense GEPP --

def test_dense_solve_exact_rational():
    rng = np.random.default_rng(1)
    for n in (1, 2, 5, 9):
        A = rng.integers(-5, 6, (n, n)).astype(float)
        A += np.eye(n) * 0.0
        while abs(np.linalg.det(A)) < 0.5:
            A = rng.integers(-5, 6, (n, n)).astype(float)
        b = rng.integers(-9, 10, n).astype(float)
        xe = np.array([float(v) for v in _gepp_fraction(A, b)])
        x = oracle.dense_solve(A, b)
        assert np.allclose(x, xe, rtol=1e-12, atol=1e-12)


def test_dense_solve_needs_pivoting():
    A = np.array([[0.0, 1.0, 2.0], [1.0, 0.0, 3.0], [4.0, -3.0, 8.0]])
    b = np.array([1.0, 2.0, 3.0])
    assert np.allclose(oracle.dense_solve(A, b), np.linalg.solve(A, b), rtol=1e-14)
    with pytest.raises(oracle.SingularError):
        oracle.dense_solve(np.array([[1.0, 2.0], [2.0, 4.0]]), np.ones(2))


# ----------------------------------------------------- scalar tridiagonal --

def _poisson_exact(fint):
    """x = A^{-1} f for tridiag(-1,2,-1), from (A^{-1})_{ij} = min(i,j)(n+1-max(i,j))/(n+1)
    (1-based), in exact integer arithmetic; returns numerators over (n+1)."""
    n = len(fint)
    i1 = np.arange(1, n + 1, dtype=object)
    f = np.array([int(v) for v in fint], dtype=object)
    left = np.cumsum(i1 * f)                         # sum_{j<=i} j f_j
    right_terms = (n + 1 - i1) * f
    right = np.concatenate([np.cumsum(right_terms[::-1])[::-1][1:], np.array([0], dtype=object)])
    return (n + 1 - i1) * left + i1 * right, n + 1


@pytest.mark.parametrize("n", [1, 2, 7, 64, 4096])
def test_tri_poisson_closed_form(n):
    dl, d, du = gen.poisson(n)
    rng = np.random.default_rng(n)
    fint = rng.integers(-3, 4, n)
    fint[0] = 3                                      # never the zero vector
    num, den = _poisson_exact(fint)
    xe = np.array([Fraction(int(v), den) for v in num], dtype=object)
    xe_f = np.array([float(v) for v in xe])
    x = oracle.tri_solve(dl, d, du, fint.astype(float))
    # kappa_2 from the closed-form eigenvalues 2 - 2 cos(k pi/(n+1))
    lam = 2 - 2 * np.cos(np.arange(1, n + 1) * np.pi / (n + 1))
    kappa = lam.max() / lam.min()
    err = np.linalg.norm(x - xe_f) / max(np.linalg.norm(xe_f), 1e-300)
    assert err <= 10 * kappa * np.finfo(float).eps
    # backward error ||f - A x|| / (||A|| ||x|| + ||f||)
    r = oracle.tri_residual(dl, d, du, x, fint.astype(float))
    bwd = np.linalg.norm(r) / (4 * np.linalg.norm(x) + np.linalg.norm(fint))
    assert bwd <= 1e-14


@pytest.mark.parametrize("n", [1, 3, 100, 4096])
def test_tri_poisson_f_equal_2(n):
    """f = 2 everywhere has the exact solution x_i = i (n+1-i)."""
    dl, d, du = gen.poisson(n)
    x = oracle.tri_solve(dl, d, du, 2.0 * np.ones(n))
    i = np.arange(1, n + 1, dtype=float)
    xe = i * (n + 1 - i)
    lam = 2 - 2 * np.cos(np.arange(1, n + 1) * np.pi / (n + 1))
    kappa = lam.max() / lam.min()
    assert np.linalg.norm(x - xe) / np.linalg.norm(xe) <= 10 * kappa * np.finfo(float).eps


@pytest.mark.parametrize("n,nrhs", [(1, 1), (2, 3), (17, 2), (512, 4)])
def test_tri_vs_dense_lapack(n, nrhs):
    s = gen.tri_sdd(n, nrhs, seed_rep=n)
    A = np.diag(s.d) + np.diag(s.dl[1:], -1) + np.diag(s.du[:-1], 1)
    xr = np.linalg.solve(A, s.f)
    x = oracle.tri_solve(s.dl, s.d, s.du, s.f)
    assert oracle.rel_err(x, xr) <= 1e-14
    assert oracle.rel_err(x, s.xstar) <= 1e-14


def test_tri_residual_matches_dense():
    s = gen.tri_sdd(50, 2)
    A = np.diag(s.d) + np.diag(s.dl[1:], -1) + np.diag(s.du[:-1], 1)
    x = np.random.default_rng(0).standard_normal((50, 2))
    assert np.allclose(oracle.tri_residual(s.dl, s.d, s.du, x, s.f), s.f - A @ x, atol=1e-13)


def test_tri_singular_detected():
    with pytest.raises(oracle.SingularError):
        oracle.tri_solve(np.array([0.0, 1.0]), np.array([1.0, 1.0]), np.array([1.0, 0.0]), np.ones(2))


# ------------------------------------------------------- block tridiagonal --

@pytest.mark.parametrize("N,m,nrhs", [(1, 3, 1), (2, 2, 2), (9, 4, 3), (40, 8, 2), (12, 16, 1), (6, 32, 2)])
def test_btri_vs_dense_lapack(N, m, nrhs):
    s = gen.btri_random(N, m, nrhs, seed_rep=N * 100 + m)
    A = gen.btri_dense(s.B, s.D, s.C)
    Xr = np.linalg.solve(A, s.F)
    X = oracle.btri_solve(s.B, s.D, s.C, s.F)
    assert oracle.rel_err(X, Xr) <= 1e-13
    R = oracle.btri_residual(s.B, s.D, s.C, X, s.F)
    assert np.allclose(R, s.F - A @ X, atol=1e-12)


def test_btri_block_diagonal_reduces_to_independent_solves():
    s = gen.btri_random(7, 5, 2)
    Z = np.zeros_like(s.B)
    X = oracle.btri_solve(Z, s.D, Z, s.F).reshape(7, 5, 2)
    for j in range(7):
        assert np.allclose(X[j], np.linalg.solve(s.D[j], s.F.reshape(7, 5, 2)[j]), rtol=1e-13, atol=1e-14)


def test_btri_m1_equals_scalar_thomas():
    s = gen.tri_sdd(300, 2)
    X = oracle.btri_solve(s.dl.reshape(-1, 1, 1), s.d.reshape(-1, 1, 1), s.du.reshape(-1, 1, 1), s.f)
    x = oracle.tri_solve(s.dl, s.d, s.du, s.f)
    # the two differ only in rounding order (h - Y x vs (g - du x)/u)
    assert oracle.rel_err(X, x) <= 1e-15


def test_btri_pivoting_inside_blocks():
    """Diagonal blocks with a zero leading entry need the in-block pivoting."""
    N, m = 5, 3
    rng = np.random.default_rng(3)
    P = np.array([[0.0, 1.0, 0.0], [1.0, 0.0, 0.0], [0.0, 0.0, 1.0]])
    D = np.stack([4.0 * P + 0.1 * rng.standard_normal((m, m)) for _ in range(N)])
    for j in range(N):
        D[j, 0, 0] = 0.0
    B = 0.3 * rng.standard_normal((N, m, m))
    C = 0.3 * rng.standard_normal((N, m, m))
    B[0] = 0
    C[-1] = 0
    F = rng.standard_normal((N * m, 2))
    X = oracle.btri_solve(B, D, C, F)
    assert oracle.rel_err(X, np.linalg.solve(gen.btri_dense(B, D, C), F)) <= 1e-13


# -------------------------------------------------------------------- BABD --

@pytest.mark.parametrize("N,m,nrhs,sep", [(1, 2, 1, False), (3, 4, 2, False), (20, 8, 3, False),
                                          (17, 8, 1, True), (30, 3, 2, True), (9, 16, 1, False)])
def test_babd_vs_dense_lapack(N, m, nrhs, sep):
    b = gen.babd_bvp(N, m, nrhs, separated=sep, seed_rep=N + m)
    A = gen.babd_dense(b.S, b.R, b.B0, b.B1)
    Yr = np.linalg.solve(A, b.RHS)
    Y = oracle.babd_solve(b.S, b.R, b.B0, b.B1, b.RHS)
    assert oracle.rel_err(Y, Yr) <= 1e-12
    R = oracle.babd_residual(b.S, b.R, b.B0, b.B1, Y, b.RHS)
    assert np.allclose(R, b.RHS - A @ Y, atol=1e-12)


def test_babd_generic_vs_dense():
    b = gen.babd_random(25, 6, 2)
    A = gen.babd_dense(b.S, b.R, b.B0, b.B1)
    Y = oracle.babd_solve(b.S, b.R, b.B0, b.B1, b.RHS)
    assert oracle.rel_err(Y, np.linalg.solve(A, b.RHS)) <= 1e-13
    assert oracle.rel_err(Y, b.Yexact) <= 1e-12


def test_babd_ivp_special_case_is_time_stepping():
    """B0 = I, B1 = 0 makes the BABD system the initial value problem of
    Sec. 3; its solution is the sequential recurrence of Eq. (My):
    y_0 = beta, R_j y_{j+1} = r_j - S_j y_j."""
    N, m = 64, 4
    b = gen.babd_bvp(N, m, 2)
    B0 = np.eye(m)
    B1 = np.zeros((m, m))
    RHS = b.RHS.copy()
    Y = oracle.babd_solve(b.S, b.R, B0, B1, RHS).reshape(N + 1, m, 2)
    Rb = RHS.reshape(N + 1, m, 2)
    y = Rb[0].copy()
    ref = [y]
    for j in range(N):
        y = np.linalg.solve(b.R[j], Rb[j + 1] - b.S[j] @ y)
        ref.append(y)
    assert oracle.rel_err(Y, np.stack(ref)) <= 1e-13


def test_babd_trapezoidal_second_order():
    """The discrete solution converges to y(t) = exp(sin 3t) v at order 2:
    the max error falls by about 4 per halving of h."""
    prob = gen.bvp_problem(8, 1, seed_rep=0)
    errs = []
    Ns = [2 ** k for k in range(6, 12)]
    for N in Ns:
        b = gen.trapezoidal_babd(prob, N)
        Y = oracle.babd_solve(b.S, b.R, b.B0, b.B1, b.RHS)
        errs.append(np.abs(Y - b.Yexact).max())
    ratios = [errs[i] / errs[i + 1] for i in range(len(errs) - 1)]
    assert all(3.6 < r < 4.4 for r in ratios), ratios
    orders = np.log2(ratios)
    assert abs(np.mean(orders) - 2.0) < 0.05


def test_babd_separated_bc_singular_b0():
    """Separated boundary conditions: B0 and B1 are both singular, so the
    boundary row needs pivoting against later rows."""
    b = gen.babd_bvp(160, 8, 1, separated=True)
    assert np.linalg.matrix_rank(b.B0) < 8 and np.linalg.matrix_rank(b.B1) < 8
    Y = oracle.babd_solve(b.S, b.R, b.B0, b.B1, b.RHS)
    A = gen.babd_dense(b.S, b.R, b.B0, b.B1)
    assert oracle.rel_err(Y, np.linalg.solve(A, b.RHS)) <= 1e-12
    assert np.abs(Y - b.Yexact).max() < 1e-2
