"""Parareal (Secs. 3-4: the iterative solution of the IVP reduced system with a
coarse propagator) on the GPU against the oracle's plain iteration: every
iterate element by element, convergence to the sequential fine solution, and
a large problem checked against the oracle's sequential integration."""
import numpy as np
import pytest

from oracle import ivp
from conftest import to_dev, to_host

pytestmark = pytest.mark.gpu


def _problem(n, seed):
    dl, d, du = ivp.laplacian(n, nu=0.5)
    rng = np.random.default_rng(seed)
    y0 = rng.standard_normal(n)
    g0 = rng.standard_normal(n)
    g1 = rng.standard_normal(n)
    return dl, d, du, y0, g0, g1


@pytest.mark.parametrize("n,p,nfine,ncoarse", [(1, 3, 4, 1), (64, 8, 10, 2), (257, 32, 5, 1), (100, 5, 1, 3)])
def test_parareal_iterates_match_oracle(cuda, n, p, nfine, ncoarse):
    import paper_0912_3678_gb300 as bt
    dl, d, du, y0, g0, g1 = _problem(n, n + p)
    T = 0.05
    ref = ivp.parareal(dl, d, du, y0, g0, g1, T, p, nfine, ncoarse, p)
    U, it, code, hist = bt.ivp_parareal(*(to_dev(a, cuda) for a in (dl, d, du, g0, y0)), T, p, nfine, ncoarse,
                                        kmax=p, tol=0.0, g1=to_dev(g1, cuda), keep_history=True)
    assert it == p
    H = to_host(hist)
    scale = np.abs(ref).max()
    for k in range(p + 1):
        assert np.abs(H[k] - ref[k]).max() <= 1e-12 * scale, k
    seq = ivp.sequential_fine(dl, d, du, y0, g0, g1, T, p, nfine)
    assert np.abs(to_host(U) - seq).max() <= 1e-12 * scale


def test_parareal_stops_on_tolerance(cuda):
    import paper_0912_3678_gb300 as bt
    n, p, nfine = 128, 16, 20
    dl, d, du, y0, g0, g1 = _problem(n, 3)
    T = 0.1
    U, it, code, _ = bt.ivp_parareal(*(to_dev(a, cuda) for a in (dl, d, du, g0, y0)), T, p, nfine, 1,
                                     kmax=p, tol=1e-10, g1=to_dev(g1, cuda))
    assert code == 0 and 1 <= it < p
    seq = ivp.sequential_fine(dl, d, du, y0, g0, g1, T, p, nfine)
    assert np.abs(to_host(U) - seq).max() <= 1e-8 * np.abs(seq).max()
    U2, it2, code2, _ = bt.ivp_parareal(*(to_dev(a, cuda) for a in (dl, d, du, g0, y0)), T, p, nfine, 1,
                                        kmax=1, tol=1e-14, g1=to_dev(g1, cuda), raise_on_error=False)
    assert code2 == 5 and it2 == 1          # BT_ERR_NOT_CONVERGED after kmax iterations


def test_parareal_large_problem(cuda):
    """n = 2^17 unknowns, 16 intervals of 12 trapezoidal steps: after p
    iterations the coarse values equal the oracle's sequential integration."""
    import paper_0912_3678_gb300 as bt
    n, p, nfine = 1 << 17, 16, 12
    dl, d, du, y0, g0, g1 = _problem(n, 7)
    T = 1e-4
    U, it, code, _ = bt.ivp_parareal(*(to_dev(a, cuda) for a in (dl, d, du, g0, y0)), T, p, nfine, 2,
                                     kmax=p, tol=0.0, g1=to_dev(g1, cuda))
    seq = ivp.sequential_fine(dl, d, du, y0, g0, g1, T, p, nfine)
    assert np.abs(to_host(U) - seq).max() <= 1e-11 * np.abs(seq).max()


def test_parareal_invalid_arguments(cuda):
    import paper_0912_3678_gb300 as bt
    dl, d, du, y0, g0, g1 = _problem(16, 1)
    args = [to_dev(a, cuda) for a in (dl, d, du, g0, y0)]
    for bad in (dict(p=33, nfine=2), dict(p=0, nfine=2), dict(p=4, nfine=0)):
        with pytest.raises(bt.BtError):
            bt.ivp_parareal(*args, 0.1, bad["p"], bad["nfine"], 1)
    with pytest.raises(bt.BtError):
        bt.ivp_parareal(*args, -1.0, 4, 2, 1)


# ------------------------------------------------------------------ block BVM --
def _bvm_problem(m, p, N, T, seed):
    rng = np.random.default_rng(seed)
    Q, _ = np.linalg.qr(rng.standard_normal((m, m)))
    L = Q @ np.diag(-rng.uniform(0.5, 3.0, m)) @ Q.T + 0.1 * rng.standard_normal((m, m))
    v = rng.standard_normal(m)
    y = lambda t: np.exp(np.sin(3 * t)) * v
    dy = lambda t: 3 * np.cos(3 * t) * np.exp(np.sin(3 * t)) * v
    t = np.arange(p * N + 1) * (T / (p * N))
    G = np.array([dy(tk) - L @ y(tk) for tk in t])
    return L, y(0.0), G, np.array([y(tk) for tk in t])


@pytest.mark.parametrize("m,p,N", [(1, 1, 1), (1, 3, 2), (3, 4, 7), (8, 16, 64), (16, 40, 50), (5, 33, 9)])
def test_ivp_bvm_matches_sequential_oracle(cuda, m, p, N):
    """The parallel solver (one factorization of M, the local solves (D),
    the reduced recurrence and the parallel updates) against the oracle's
    sequential recursion M_i y_i = g_i + v_i y_{N,i-1}, entry by entry; more
    than 32 intervals take several solves of at most 32 right-hand sides."""
    import paper_0912_3678_gb300 as bt
    T = 1.0
    L, y0, G, _ = _bvm_problem(m, p, N, T, seed=m + p + N)
    ref = ivp.bvm_sequential(L, y0, G, T, p, N)
    Y = bt.ivp_bvm(to_dev(L, cuda), to_dev(y0, cuda), to_dev(G, cuda), T, p, N)
    Yh = to_host(Y)
    assert np.abs(Yh - ref).max() <= 1e-12 * np.abs(ref).max()


def test_ivp_bvm_third_order_on_the_gpu(cuda):
    """The GPU solution converges to the exact y(t) with order 3."""
    import paper_0912_3678_gb300 as bt
    m, p, T = 6, 8, 1.0
    errs = []
    for N in (16, 32, 64):
        L, y0, G, exact = _bvm_problem(m, p, N, T, seed=11)
        Y = to_host(bt.ivp_bvm(to_dev(L, cuda), to_dev(y0, cuda), to_dev(G, cuda), T, p, N))
        errs.append(np.abs(Y - exact).max())
    for a, b in zip(errs, errs[1:]):
        assert 7.0 < a / b < 9.0, errs


def test_ivp_bvm_rejects_bad_arguments(cuda):
    import paper_0912_3678_gb300 as bt
    L, y0, G, _ = _bvm_problem(2, 2, 3, 1.0, seed=1)
    Ld, yd, Gd = (to_dev(a, cuda) for a in (L, y0, G))
    with pytest.raises(bt.BtError):
        bt.ivp_bvm(Ld, yd, Gd, -1.0, 2, 3)
    with pytest.raises(bt.BtError):
        bt.ivp_bvm(Ld, yd, Gd, 1.0, 0, 3)
