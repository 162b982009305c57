"""Circulant-like block systems (cyc_*, Sec. 2: after a row permutation they
take the BABD corner form): against the oracle's dense GEPP, against the
oracle's BABD elimination on the periodic BVP written with y_N as a separate
unknown and y_0 - y_N = 0, and against the periodic exact solution."""
import numpy as np
import pytest

import gen
import oracle
from conftest import to_dev, to_host

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("m", [1, 2, 4, 8, 16])
@pytest.mark.parametrize("N,nrhs", [(2, 1), (3, 2), (50, 3), (401, 1)])
def test_cyclic_matches_dense_gepp(cuda, m, N, nrhs):
    import paper_0912_3678_gb300 as bt
    s = gen.cyc_random(N, m, nrhs, seed_rep=N + m)
    ref = oracle.dense_solve(gen.cyc_dense(s.S, s.R), s.RHS)
    with bt.CycPlan(N, m, nrhs) as plan:
        plan.factor(to_dev(s.S, cuda), to_dev(s.R, cuda))
        Y = to_host(plan.solve(to_dev(s.RHS, cuda)))
        plan.sync()
    assert oracle.rel_err(Y, ref) <= 1e-11


def test_cyclic_residual_in_original_order(cuda):
    import paper_0912_3678_gb300 as bt
    N, m = 37, 4
    s = gen.cyc_random(N, m, 2, seed_rep=1)
    Y = np.random.default_rng(2).standard_normal(s.RHS.shape)
    ref = s.RHS - gen.cyc_matvec(s.S, s.R, Y)
    with bt.CycPlan(N, m, 2) as plan:
        plan.factor(to_dev(s.S, cuda), to_dev(s.R, cuda))
        Rr = to_host(plan.residual(to_dev(s.RHS, cuda), to_dev(Y, cuda)))
    assert np.abs(Rr - ref).max() <= 1e-13 * (np.abs(s.RHS).max() + 8 * np.abs(Y).max())


@pytest.mark.parametrize("prec", ["fp64", "fp32_ir"])
def test_periodic_bvp(cuda, prec):
    """y' = L(t) y + q, y(0) = y(1), trapezoidal rule, m = 8, N = 4096: equals
    the oracle's BABD elimination of the same discretisation with y_N kept as
    an unknown (B0 = I, B1 = -I, beta = 0), and the periodic exact solution to
    O(h^2)."""
    import paper_0912_3678_gb300 as bt
    N, m = 4096, 8
    s = gen.periodic_bvp(N, m, 2, seed_rep=3)
    RHSb = np.concatenate([np.zeros((m, 2)), s.RHS])
    ref = oracle.babd_solve(s.S, s.R, np.eye(m), -np.eye(m), RHSb)[:N * m]
    with bt.CycPlan(N, m, 2, prec=prec) as plan:
        plan.factor(to_dev(s.S, cuda), to_dev(s.R, cuda))
        if prec == "fp64":
            Y = to_host(plan.solve(to_dev(s.RHS, cuda)))
            plan.sync()
        else:
            Yd, it, rc, code = plan.refine(to_dev(s.RHS, cuda), tol=1e-12, maxit=20)
            assert code == 0
            Y = to_host(Yd)
    assert oracle.rel_err(Y, ref) <= (1e-11 if prec == "fp64" else 1e-10)
    assert np.abs(Y - s.Ystar).max() <= 50.0 / N ** 2 * np.abs(s.Ystar).max()


def test_cyclic_needs_two_rows(cuda):
    import paper_0912_3678_gb300 as bt
    with pytest.raises(bt.BtError):
        bt.CycPlan(1, 4, 1)
