"""Block orders outside {1,2,4,8,16,32} (embedded with an identity tail) and
banded matrices (Sec. 2: a band of s lower and r upper diagonals is block
tridiagonal with blocks of order max(s, r)), checked against the oracle."""
import numpy as np
import pytest

import gen
import oracle
from conftest import to_dev, to_host

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("m", [3, 5, 6, 7, 12, 20, 31])
@pytest.mark.parametrize("prec", ["fp64", "fp32_ir"])
def test_btri_general_block_order(cuda, m, prec):
    import paper_0912_3678_gb300 as bt
    N = 257
    s = gen.btri_random(N, m, 2, seed_rep=m)
    ref = oracle.btri_solve(s.B, s.D, s.C, s.F)
    B, D, C, F = (to_dev(a, cuda) for a in (s.B, s.D, s.C, s.F))
    with bt.BtPlan(N, m, 2, prec=prec) as plan:
        plan.factor(B, D, C)
        if prec == "fp64":
            X = plan.solve(F)
            plan.sync()
            assert oracle.rel_err(to_host(X), ref) <= 1e-11
            R = to_host(plan.residual(F, X))
            assert np.allclose(R, oracle.btri_residual(s.B, s.D, s.C, to_host(X), s.F), atol=1e-13)
        else:
            X, it, rc, code = plan.refine(F, tol=1e-12)
            assert code == 0 and oracle.rel_err(to_host(X), ref) <= 1e-10


@pytest.mark.parametrize("m", [3, 6, 12])
def test_babd_general_block_order(cuda, m):
    import paper_0912_3678_gb300 as bt
    b = gen.babd_bvp(500, m, 2, separated=(m % 2 == 0), seed_rep=m)
    ref = oracle.babd_solve(b.S, b.R, b.B0, b.B1, b.RHS)
    with bt.AbdPlan(500, m, 2) as plan:
        plan.factor(*(to_dev(a, cuda) for a in (b.S, b.R, b.B0, b.B1)))
        Y = plan.solve(to_dev(b.RHS, cuda))
        plan.sync()
    assert oracle.rel_err(to_host(Y), ref) <= 1e-11


def _band(n, s, r, rng):
    band = np.zeros((s + r + 1, n))
    A = np.zeros((n, n))
    for i in range(n):
        for k in range(max(0, i - s), min(n, i + r + 1)):
            v = rng.uniform(-1, 1) if i != k else rng.uniform(2 * (s + r) + 1, 2 * (s + r) + 3)
            band[r + i - k, k] = v
            A[i, k] = v
    return band, A


@pytest.mark.parametrize("s,r", [(1, 1), (2, 3), (5, 5), (7, 2), (0, 4)])
def test_banded_matches_dense_solve(cuda, s, r):
    import paper_0912_3678_gb300 as bt
    n = 999
    rng = np.random.default_rng(10 * s + r)
    band, A = _band(n, s, r, rng)
    f = rng.standard_normal((n, 2))
    ref = oracle.dense_solve(A, f)
    m = max(s, r, 1)
    B, D, C = bt.band_to_blocks(to_dev(band, cuda), s, r)
    N = B.shape[0]
    fp = np.zeros((N * m, 2))
    fp[:n] = f
    with bt.BtPlan(N, m, 2) as plan:
        plan.factor(B, D, C)
        X = to_host(plan.solve(to_dev(fp, cuda)))
        plan.sync()
    if X.shape[0] > n:
        assert np.abs(X[n:]).max() == 0.0      # padded unknowns
    assert oracle.rel_err(X[:n], ref) <= 1e-11


def test_padded_plan_capture(cuda):
    import paper_0912_3678_gb300 as bt
    N, m = 300, 5
    s = gen.btri_random(N, m, 1, seed_rep=99)
    B, D, C, F = (to_dev(a, cuda) for a in (s.B, s.D, s.C, s.F))
    with bt.BtPlan(N, m, 1) as plan:
        plan.factor(B, D, C)
        X = plan.solve(F)
        plan.capture("factor_solve", F, X)
        s.D = s.D + 0.5 * np.eye(m)
        D.copy_(to_dev(s.D, cuda))
        plan.replay()
        plan.sync()
    assert oracle.rel_err(to_host(X), oracle.btri_solve(s.B, s.D, s.C, s.F)) <= 1e-11
