"""Pins of the IVP / Parareal oracle (oracle/ivp.py) against closed forms and
the algebraic properties of the iteration, on the CPU."""
import numpy as np

from oracle import ivp


def _trap_factor(z):
    return (1.0 + z / 2.0) / (1.0 - z / 2.0)


def test_fine_propagator_matches_eigen_closed_form():
    """Heat equation without forcing: each eigencomponent of y0 is multiplied
    by the trapezoidal amplification factor R(h lambda_k) per step."""
    n, nsteps, h = 63, 40, 2e-3
    dl, d, du = ivp.laplacian(n)
    lam, V = ivp.eig_laplacian(n)
    rng = np.random.default_rng(1)
    c = rng.standard_normal(n)
    y0 = V @ c
    y = ivp.fine(dl, d, du, y0, np.zeros(n), None, 0.0, h, nsteps)
    exact = V @ (c * _trap_factor(h * lam) ** nsteps)
    assert np.abs(y - exact).max() <= 1e-12 * np.abs(y0).max()


def test_coarse_propagator_matches_eigen_closed_form():
    n, H, K = 31, 0.05, 3
    dl, d, du = ivp.laplacian(n)
    lam, V = ivp.eig_laplacian(n)
    c = np.random.default_rng(2).standard_normal(n)
    y = ivp.coarse(dl, d, du, V @ c, np.zeros(n), None, 0.0, H, K)
    exact = V @ (c / (1.0 - (H / K) * lam) ** K)
    assert np.abs(y - exact).max() <= 1e-12 * np.abs(c).max()


def test_steady_state_is_invariant():
    """With constant forcing g0 the steady state y* = -L^{-1} g0 is a fixed
    point of both propagators."""
    n = 40
    dl, d, du = ivp.laplacian(n)
    g0 = np.random.default_rng(3).standard_normal(n)
    A = np.diag(d) + np.diag(dl[1:], -1) + np.diag(du[:-1], 1)
    ys = -np.linalg.solve(A, g0)
    yf = ivp.fine(dl, d, du, ys, g0, None, 0.3, 1e-3, 25)
    yc = ivp.coarse(dl, d, du, ys, g0, None, 0.3, 0.1, 2)
    assert np.abs(yf - ys).max() <= 1e-10 * np.abs(ys).max()
    assert np.abs(yc - ys).max() <= 1e-10 * np.abs(ys).max()


def test_affine_forcing_matches_quadrature_of_the_trapezoidal_rule():
    """For a 1x1 system y' = a y + g0 + t g1 the trapezoidal step is the scalar
    recurrence written out by hand."""
    a, g0, g1, h, N, y = -3.0, 0.7, -1.3, 0.01, 17, 0.4
    dl, d, du = np.zeros(1), np.array([a]), np.zeros(1)
    got = ivp.fine(dl, d, du, np.array([y]), np.array([g0]), np.array([g1]), 0.25, h, N)[0]
    t = 0.25
    for _ in range(N):
        y = ((1 + h * a / 2) * y + h / 2 * ((g0 + g1 * t) + (g0 + g1 * (t + h)))) / (1 - h * a / 2)
        t += h
    assert abs(got - y) <= 1e-14


def test_parareal_properties():
    """k = 0 is the sequential coarse sweep; the iterate is exact (equal to
    the sequential fine solution) on tau_0..tau_k after k iterations, and on
    all coarse points after p iterations."""
    n, p, nfine, ncoarse, T = 24, 6, 10, 1, 0.2
    dl, d, du = ivp.laplacian(n)
    rng = np.random.default_rng(4)
    y0 = rng.standard_normal(n)
    g0 = rng.standard_normal(n)
    g1 = rng.standard_normal(n)
    U = ivp.parareal(dl, d, du, y0, g0, g1, T, p, nfine, ncoarse, p)
    ref = ivp.sequential_fine(dl, d, du, y0, g0, g1, T, p, nfine)
    H = T / p
    seqc = [y0]
    for i in range(p):
        seqc.append(ivp.coarse(dl, d, du, seqc[-1], g0, g1, i * H, H, ncoarse))
    assert np.abs(U[0] - np.array(seqc)).max() <= 1e-13 * np.abs(U[0]).max()
    scale = np.abs(ref).max()
    for k in range(p + 1):
        assert np.abs(U[k][:k + 1] - ref[:k + 1]).max() <= 1e-12 * scale
    assert np.abs(U[p] - ref).max() <= 1e-12 * scale
    # and the iteration contracts for this dissipative problem
    errs = [np.abs(U[k] - ref).max() for k in range(p + 1)]
    assert errs[2] < 0.1 * errs[0]


# ---------------------------------------------------------------- block BVM --
def _stable_L(m, seed):
    rng = np.random.default_rng(seed)
    Q, _ = np.linalg.qr(rng.standard_normal((m, m)))
    return Q @ np.diag(-rng.uniform(0.5, 3.0, m)) @ Q.T + 0.1 * rng.standard_normal((m, m))


def _forcing(L, y, dy, T, p, N):
    """g(t) = y'(t) - L y(t) at the p N + 1 fine grid points."""
    t = np.arange(p * N + 1) * (T / (p * N))
    return np.array([dy(tk) - L @ y(tk) for tk in t]), t


def test_bvm_exact_on_quadratic_solutions():
    """Both formulas (the order-3 main formula and the trapezoidal final one)
    are exact for polynomials of degree <= 2, so with g = y' - L y the
    discrete solution of (My) equals y(t) at every grid point, across the
    interval boundaries (y_{0i} = y_{N,i-1})."""
    m, p, N, T = 3, 4, 6, 1.3
    L = _stable_L(m, 1)
    c = np.random.default_rng(2).standard_normal((3, m))
    y = lambda t: c[0] + c[1] * t + c[2] * t * t
    dy = lambda t: c[1] + 2 * c[2] * t
    G, t = _forcing(L, y, dy, T, p, N)
    Y = ivp.bvm_sequential(L, y(0.0), G, T, p, N)
    ref = np.array([y(tk) for tk in t])
    assert np.abs(Y - ref).max() <= 1e-13 * np.abs(ref).max()


def test_bvm_third_order_convergence():
    """On a smooth manufactured solution the error at the grid points falls by
    about 8 per halving of h (order 3; the lower-order final formula at the
    end of each interval does not reduce it)."""
    m, p, T = 4, 2, 1.0
    L = _stable_L(m, 3)
    v = np.random.default_rng(4).standard_normal(m)
    y = lambda t: np.exp(np.sin(3 * t)) * v
    dy = lambda t: 3 * np.cos(3 * t) * np.exp(np.sin(3 * t)) * v
    errs = []
    for N in (16, 32, 64):
        G, t = _forcing(L, y, dy, T, p, N)
        Y = ivp.bvm_sequential(L, y(0.0), G, T, p, N)
        errs.append(np.abs(Y - np.array([y(tk) for tk in t])).max())
    for a, b in zip(errs, errs[1:]):
        assert 7.0 < a / b < 9.0, errs
