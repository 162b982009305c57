"""GPU parity of the BABD partition solver (abd_*) against the oracle."""
import numpy as np
import pytest

import gen
import oracle
from oracle import partition as P
from conftest import to_dev, to_host

pytestmark = pytest.mark.gpu


def _solve(cuda, b, p=0, prec="fp64"):
    import paper_0912_3678_gb300 as bt
    N, m = b.S.shape[0], b.S.shape[1]
    nr = b.RHS.shape[1]
    with bt.AbdPlan(N, m, nrhs_max=nr, prec=prec, p=p) as plan:
        plan.factor(*(to_dev(a, cuda) for a in (b.S, b.R, b.B0, b.B1)))
        Y = plan.solve(to_dev(b.RHS, cuda))
        plan.sync()
        return to_host(Y), plan.levels()


@pytest.mark.parametrize("m", [1, 2, 4, 8, 16, 32])
@pytest.mark.parametrize("N,nrhs,sep", [(1, 1, False), (5, 2, False), (9, 1, True), (100, 3, False),
                                        (777, 1, True)])
def test_babd_fp64_matches_oracle(cuda, m, N, nrhs, sep):
    if sep and m == 1:
        pytest.skip("separated conditions need m >= 2")
    b = gen.babd_bvp(N, m, nrhs, separated=sep, seed_rep=N + m)
    Y, lev = _solve(cuda, b)
    ref = oracle.babd_solve(b.S, b.R, b.B0, b.B1, b.RHS)
    assert oracle.rel_err(Y, ref) <= 1e-11, lev


@pytest.mark.parametrize("m", [4, 8, 16])
@pytest.mark.parametrize("p", [1, 2, 3, 10, 49])
def test_babd_invariant_under_p(cuda, p, m):
    b = gen.babd_random(100, m, 2, seed_rep=1)
    Y, _ = _solve(cuda, b, p=p)
    ref = oracle.babd_solve(b.S, b.R, b.B0, b.B1, b.RHS)
    assert oracle.rel_err(Y, ref) <= 1e-11


def test_babd_reduced_matrix(cuda):
    import paper_0912_3678_gb300 as bt
    b = gen.babd_bvp(40, 4, 1, seed_rep=5)
    al, be, g, T = P.babd_reduced_blocks(b.S, b.R, b.B0, b.B1, b.RHS, 5)
    with bt.AbdPlan(40, 4, 1, p=5) as plan:
        plan.factor(*(to_dev(a, cuda) for a in (b.S, b.R, b.B0, b.B1)))
        a_, b_ = (to_host(t) for t in plan.reduced())
    scale = np.abs(T).max()
    assert np.abs(a_ - al).max() <= 1e-13 * scale
    assert np.abs(b_ - be).max() <= 1e-13 * scale


def test_babd_m8_n262144_full_size(cuda):
    """Trapezoidal BABD, m = 8, N = 2^18 steps: parity with the oracle and the
    O(h^2) error against the exact solution y(t) = exp(sin 3t) v."""
    N = 1 << 18
    b = gen.babd_bvp(N, 8, 1, seed_rep=0)
    Y, lev = _solve(cuda, b)
    ref = oracle.babd_solve(b.S, b.R, b.B0, b.B1, b.RHS)
    assert oracle.rel_err(Y, ref) <= 1e-11
    h = 1.0 / N
    assert np.abs(Y - b.Yexact).max() <= 200 * h * h


def test_babd_m8_n262144_separated_full_size(cuda):
    N = 1 << 18
    b = gen.babd_bvp(N, 8, 1, separated=True, seed_rep=1)
    Y, lev = _solve(cuda, b)
    ref = oracle.babd_solve(b.S, b.R, b.B0, b.B1, b.RHS)
    assert oracle.rel_err(Y, ref) <= 1e-11


def test_babd_mixed_precision_refinement(cuda):
    import paper_0912_3678_gb300 as bt
    b = gen.babd_bvp(5000, 8, 2, seed_rep=3)
    ref = oracle.babd_solve(b.S, b.R, b.B0, b.B1, b.RHS)
    with bt.AbdPlan(5000, 8, 2, prec="fp32_ir") as plan:
        plan.factor(*(to_dev(a, cuda) for a in (b.S, b.R, b.B0, b.B1)))
        Y, it, rc, code = plan.refine(to_dev(b.RHS, cuda), tol=1e-12, maxit=20)
    assert code == 0
    assert oracle.rel_err(to_host(Y), ref) <= 1e-10


def test_babd_residual(cuda):
    import paper_0912_3678_gb300 as bt
    b = gen.babd_random(60, 8, 2, seed_rep=2)
    Yr = np.random.default_rng(1).standard_normal(b.RHS.shape)
    ref = oracle.babd_residual(b.S, b.R, b.B0, b.B1, Yr, b.RHS)
    with bt.AbdPlan(60, 8, 2) as plan:
        plan.factor(*(to_dev(a, cuda) for a in (b.S, b.R, b.B0, b.B1)))
        R = to_host(plan.residual(to_dev(b.RHS, cuda), to_dev(Yr, cuda)))
    assert np.abs(R - ref).max() <= 1e-13 * (np.abs(b.RHS).max() + 16 * np.abs(Yr).max())


def test_ivp_special_case(cuda):
    """B0 = I, B1 = 0: the time-parallel IVP solve of Sec. 3 equals sequential
    time stepping (Eq. (My))."""
    b = gen.babd_bvp(3000, 4, 1, seed_rep=6)
    b.B0 = np.eye(4)
    b.B1 = np.zeros((4, 4))
    Y, _ = _solve(cuda, b)
    Rb = b.RHS.reshape(3001, 4, 1)
    y = Rb[0].copy()
    seq = [y]
    for j in range(3000):
        y = np.linalg.solve(b.R[j], Rb[j + 1] - b.S[j] @ y)
        seq.append(y)
    assert oracle.rel_err(Y, np.concatenate(seq)) <= 1e-11


def test_babd_anorm_matches_numpy(cuda):
    import paper_0912_3678_gb300 as bt
    b = gen.babd_random(300, 8, 1, seed_rep=4)
    rows = np.concatenate([np.abs(b.B0).sum(1) + np.abs(b.B1).sum(1),
                           (np.abs(b.S).sum(2) + np.abs(b.R).sum(2)).ravel()])
    exact = rows.max()
    with bt.AbdPlan(300, 8, 1) as plan:
        plan.factor(*(to_dev(a, cuda) for a in (b.S, b.R, b.B0, b.B1)))
        got = plan.anorm()
    assert abs(got - exact) <= 1e-5 * exact


@pytest.mark.parametrize("m,N", [(4, 5000), (8, 3000)])
def test_babd_captured_step_refactors_new_matrices(cuda, m, N):
    """Captured factor+solve of a BABD plan (reduced-system levels factored on a
    second stream beside the level-0 forward substitution), replayed after the
    blocks and right-hand side are overwritten in place: the new system's
    solution."""
    import paper_0912_3678_gb300 as bt
    b0 = gen.babd_random(N, m, 2, seed_rep=5)
    b1 = gen.babd_random(N, m, 2, seed_rep=6)
    S, R, B0, B1, F = (to_dev(a, cuda) for a in (b0.S, b0.R, b0.B0, b0.B1, b0.RHS))
    with bt.AbdPlan(N, m, nrhs_max=2) as plan:
        assert len(plan.levels()) >= 2
        plan.factor(S, R, B0, B1)
        Y = plan.solve(F)
        plan.capture("factor_solve", F, Y)
        for b in (b1, b0):
            for dev, host in zip((S, R, B0, B1, F), (b.S, b.R, b.B0, b.B1, b.RHS)):
                dev.copy_(to_dev(host, cuda))
            Y.zero_()
            plan.replay()
            plan.sync()
            ref = oracle.babd_solve(b.S, b.R, b.B0, b.B1, b.RHS)
            assert oracle.rel_err(to_host(Y), ref) <= 1e-11


@pytest.mark.parametrize("m", [2, 4])
@pytest.mark.parametrize("p", [19456, 0])
def test_babd_thread_and_lane_group_kernels(cuda, m, p):
    """BABD levels of block order 2 and 4: one thread per partition where the
    partitions fill a whole wave (p = 128 per SM), a group of m*m lanes per
    partition elsewhere (the recursion levels, and every level by default)."""
    b = gen.babd_random(50000, m, 3, seed_rep=m)
    Y, lev = _solve(cuda, b, p=p)
    ref = oracle.babd_solve(b.S, b.R, b.B0, b.B1, b.RHS)
    assert oracle.rel_err(Y, ref) <= 1e-11, lev


@pytest.mark.parametrize("m", [8, 16, 32])
@pytest.mark.parametrize("N,nrhs,sep", [(1, 1, False), (2, 2, True), (3, 1, False), (7, 3, True), (100, 2, False),
                                        (777, 1, True), (4099, 3, False)])
def test_babd_cyclic_reduction_matches_oracle(cuda, m, N, nrhs, sep):
    """Cyclic reduction of the whole BABD system (abd tuning reduced = 1): odd
    and even level sizes, separated and general boundary conditions."""
    import paper_0912_3678_gb300 as bt
    b = gen.babd_bvp(N, m, nrhs, separated=sep, seed_rep=3 * N + m)
    with bt.AbdPlan.tuned(N, m, nrhs, "fp64", {"reduced": 1}) as plan:
        plan.factor(*(to_dev(a, cuda) for a in (b.S, b.R, b.B0, b.B1)))
        Y = to_host(plan.solve(to_dev(b.RHS, cuda)))
        plan.sync()
    ref = oracle.babd_solve(b.S, b.R, b.B0, b.B1, b.RHS)
    assert oracle.rel_err(Y, ref) <= 1e-11


def test_babd_cyclic_reduction_trapezoidal_bvp_order(cuda):
    """On the manufactured trapezoidal BVP the cyclic-reduction solution meets
    the exact y(t) to second order, like the partition solution."""
    import paper_0912_3678_gb300 as bt
    errs = []
    for N in (256, 512, 1024):
        b = gen.babd_bvp(N, 8, 1, seed_rep=0)
        with bt.AbdPlan.tuned(N, 8, 1, "fp64", {"reduced": 1}) as plan:
            plan.factor(*(to_dev(a, cuda) for a in (b.S, b.R, b.B0, b.B1)))
            Y = to_host(plan.solve(to_dev(b.RHS, cuda)))
        errs.append(np.abs(Y - b.Yexact).max())
    assert 3.5 < errs[0] / errs[1] < 4.5 and 3.5 < errs[1] / errs[2] < 4.5


def test_babd_cyclic_reduction_reports_a_singular_block(cuda):
    """A zero R_{2k} (host-made fault in the input) is a singular pivot block at
    row 2k of the first level."""
    import paper_0912_3678_gb300 as bt
    b = gen.babd_random(64, 8, 1, seed_rep=2)
    b.R[10] = 0.0
    with bt.AbdPlan.tuned(64, 8, 1, "fp64", {"reduced": 1}) as plan:
        plan.factor(*(to_dev(a, cuda) for a in (b.S, b.R, b.B0, b.B1)))
        code, lev, part, row = plan.info()
    assert bt.BT_STATUS[code] == "BT_ERR_SINGULAR"
    assert (lev, row) == (0, 10)


def test_babd_cyclic_reduction_refuses_unsupported_plans(cuda):
    import paper_0912_3678_gb300 as bt
    for m, prec in ((4, "fp64"), (8, "fp32_ir"), (12, "fp64")):
        with pytest.raises(bt.BtError):
            bt.AbdPlan.tuned(100, m, 1, prec, {"reduced": 1})
