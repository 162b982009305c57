"""Pivoted partitions (bt_tuning.pivot = 1, the variant of Sec. 2 for local
blocks that are singular or ill-conditioned): local factorizations stop at a
breakdown row, which joins the reduced system; the enlarged reduced system is
solved by elimination with partial pivoting.  Checked against the oracle's
dense GEPP on systems whose diagonal blocks are often exactly singular, where
the plain partition method reports BT_ERR_SINGULAR."""
import numpy as np
import pytest

import gen
import oracle
from conftest import to_dev, to_host

pytestmark = pytest.mark.gpu


def _backward_error(s, X):
    R = oracle.btri_residual(s.B, s.D, s.C, X, s.F)
    rows = np.abs(s.D).sum(2)
    rows[1:] += np.abs(s.B[1:]).sum(2)
    rows[:-1] += np.abs(s.C[:-1]).sum(2)
    return np.abs(R).max() / (rows.max() * np.abs(X).max() + np.abs(s.F).max())


def _check(s, X, tau=1e-3):
    """Normwise backward error within 4 (3m+1) u times the multiplier bound
    1/tau of threshold pivoting (the local factorizations accept pivots down to
    tau times the row's largest entry), forward error within kappa times that,
    against the oracle's dense GEPP."""
    m = s.D.shape[1]
    A = gen.btri_dense(s.B, s.D, s.C)
    ref = oracle.dense_solve(A, s.F)
    kappa = np.linalg.cond(A, 1)
    eta = 4 * (3 * m + 1) * 2.0 ** -53 / max(tau, 1e-3)
    assert _backward_error(s, X) <= eta
    assert oracle.rel_err(X, ref) <= 1e-11 + eta * kappa


@pytest.mark.parametrize("m", [1, 2, 4, 8, 16])
@pytest.mark.parametrize("N,p0", [(64, 4), (300, 16), (301, 1)])
def test_pivoted_partitions_match_dense_gepp(cuda, m, N, p0):
    import paper_0912_3678_gb300 as bt
    s = gen.btri_nondominant(N, m, 2, seed_rep=N + 7 * m, zero_frac=0.08)
    with bt.BtPlan.tuned(N, m, 2, "fp64", {"p0": p0, "pivot": 1}) as plan:
        plan.factor(*(to_dev(a, cuda) for a in (s.B, s.D, s.C)))
        X = to_host(plan.solve(to_dev(s.F, cuda)))
        plan.sync()
        p_eff = plan.levels()[0][1]
    _check(s, X)
    assert p_eff >= p0


def test_plain_partitions_report_the_singular_block(cuda):
    """Without pivoting, an exactly singular pivot block (D_j = 0 on the first
    local row of a partition, where the pivot block is D_j itself) stops the
    plain method with BT_ERR_SINGULAR; the pivoted plan solves the system."""
    import paper_0912_3678_gb300 as bt
    N, m = 300, 4
    s = gen.btri_nondominant(N, m, 1, seed_rep=3, zero_frac=0.0)
    s.D[19] = 0.0          # partitions of 18-19 rows: partition 1 starts at row 19
    with bt.BtPlan.tuned(N, m, 1, "fp64", {"p0": 16}) as plan:
        plan.factor(*(to_dev(a, cuda) for a in (s.B, s.D, s.C)))
        code, lev, part, row = plan.info()
    assert bt.BT_STATUS[code] == "BT_ERR_SINGULAR" and row == 19
    with bt.BtPlan.tuned(N, m, 1, "fp64", {"p0": 16, "pivot": 1}) as plan:
        plan.factor(*(to_dev(a, cuda) for a in (s.B, s.D, s.C)))
        X = to_host(plan.solve(to_dev(s.F, cuda)))
        plan.sync()
    _check(s, X)


@pytest.mark.parametrize("m", [1, 8])
def test_pivoted_fp32_refined(cuda, m):
    import paper_0912_3678_gb300 as bt
    N = 400
    s = gen.btri_nondominant(N, m, 3, seed_rep=11 + m, zero_frac=0.05)
    with bt.BtPlan.tuned(N, m, 3, "fp32_ir", {"p0": 8, "pivot": 1}) as plan:
        plan.factor(*(to_dev(a, cuda) for a in (s.B, s.D, s.C)))
        X, it, rc, code = plan.refine(to_dev(s.F, cuda), tol=1e-12, maxit=40)
    assert code == 0
    _check(s, to_host(X))


def test_pivoted_reduced_matrix_is_schur_complement(cuda):
    """The enlarged reduced matrix equals the Schur complement of A onto the
    separators: the uniform ones plus the rows promoted by splits.  With
    tau = 0 only exactly singular pivot blocks break down; a zero D_j on the
    first local row of a partition (where the pivot block is D_j itself) is
    one, so the promoted rows are known in advance."""
    import paper_0912_3678_gb300 as bt
    from oracle import partition as P
    N, m = 40, 2
    s = gen.btri_nondominant(N, m, 1, seed_rep=5, zero_frac=0.0)
    s.D[5] = 0.0           # partitions of 5 rows: first local rows 0, 5, 10, ...
    s.D[20] = 0.0
    with bt.BtPlan.tuned(N, m, 1, "fp64", {"p0": 8, "pivot": 1}) as plan:
        bt.bt_plan_set_pivot_tol(plan.handle, 0.0)
        plan.factor(*(to_dev(a, cuda) for a in (s.B, s.D, s.C)))
        p_eff = plan.levels()[0][1]
        al, be, ga = (to_host(t) for t in plan.reduced())
    allseps = sorted([4, 9, 14, 19, 24, 29, 34] + [5, 20])
    assert p_eff - 1 == len(allseps)
    A = gen.btri_dense(s.B, s.D, s.C)
    bounds = [-1] + allseps + [N]
    local = [(a + 1, b) for a, b in zip(bounds[:-1], bounds[1:])]
    T, _ = P.schur_reduced(A, s.F, m, local, allseps)
    K = len(allseps)
    scale = np.abs(T).max()
    for k in range(K):
        blk = T[k * m:(k + 1) * m]
        assert np.abs(al[k] - blk[:, k * m:(k + 1) * m]).max() <= 1e-11 * scale
        if k > 0:
            assert np.abs(be[k] - blk[:, (k - 1) * m:k * m]).max() <= 1e-11 * scale
        if k + 1 < K:
            assert np.abs(ga[k] - blk[:, (k + 1) * m:(k + 2) * m]).max() <= 1e-11 * scale


def test_pivoted_breakdown_at_partition_ends(cuda):
    """Splits that leave partitions without local rows: on block row 0 (the
    first partition becomes a lone separator), on the first local row of a
    partition, and on the last two block rows (the last partition is left
    with no rows at all).  Partitions of 2 rows, tau = 0."""
    import paper_0912_3678_gb300 as bt
    N, m = 60, 4
    s = gen.btri_nondominant(N, m, 2, seed_rep=8, zero_frac=0.0)
    for r in (0, 10, 58, 59):
        s.D[r] = 0.0
    with bt.BtPlan.tuned(N, m, 2, "fp64", {"p0": 30, "pivot": 1}) as plan:
        bt.bt_plan_set_pivot_tol(plan.handle, 0.0)
        plan.factor(*(to_dev(a, cuda) for a in (s.B, s.D, s.C)))
        X = to_host(plan.solve(to_dev(s.F, cuda)))
        plan.sync()
        assert plan.levels()[0][1] == 34
    _check(s, X)


def test_pivoted_solve_graph_and_limits(cuda):
    """Solves of a pivoted plan can be captured (its factorization cannot);
    a system whose every diagonal block is singular needs more separators
    than the reduced system holds and is refused with BT_ERR_SINGULAR."""
    import paper_0912_3678_gb300 as bt
    N, m = 200, 8
    s = gen.btri_nondominant(N, m, 1, seed_rep=9, zero_frac=0.05)
    B, D, C, F = (to_dev(a, cuda) for a in (s.B, s.D, s.C, s.F))
    with bt.BtPlan.tuned(N, m, 1, "fp64", {"p0": 8, "pivot": 1}) as plan:
        plan.factor(B, D, C)
        X = F.clone().zero_()
        with pytest.raises(bt.BtError):
            plan.capture("factor_solve", F, X)
        plan.capture("solve", F, X)
        plan.replay()
        plan.sync()
        _check(s, to_host(X))
    s.D[:] = 0.0
    with bt.BtPlan.tuned(N, m, 1, "fp64", {"p0": 8, "pivot": 1}) as plan:
        with pytest.raises(bt.BtError):
            plan.factor(*(to_dev(a, cuda) for a in (s.B, s.D, s.C)))
