"""Partitions factored by local QR (bt_tuning.pivot = 2, the variant of Sec. 2
with N^(i) = Q^(i) and S^(i) = R^(i)): each partition's local block is reduced
by Householder steps, so singular or ill-conditioned diagonal blocks need no
splitting and the reduced system keeps its p-1 block rows.  Checked against
the oracle's dense GEPP solution and its Schur complement, on the
non-dominant systems of the pivoted-partition tests."""
import numpy as np
import pytest

import gen
import oracle
from conftest import to_dev, to_host
from oracle import partition as P

pytestmark = pytest.mark.gpu

U = 2.0 ** -53


def _backward_error(s, X):
    R = oracle.btri_residual(s.B, s.D, s.C, X, s.F)
    rows = np.abs(s.D).sum(2)
    rows[1:] += np.abs(s.B[1:]).sum(2)
    rows[:-1] += np.abs(s.C[:-1]).sum(2)
    return np.abs(R).max() / (rows.max() * np.abs(X).max() + np.abs(s.F).max())


def _eta(s, p):
    """Backward-error bound: 16 times the backward error of the oracle's
    partition solve by definition on the same partitions (the Schur
    complement of the local blocks, which carries their conditioning into the
    reduced system whatever the local factorization), plus 4 (3m+1) u, the
    bound of the unpivoted tests."""
    m = s.D.shape[1]
    xp = P.partition_solve(s.B, s.D, s.C, s.F, p)
    return 16 * _backward_error(s, xp) + 4 * (3 * m + 1) * U


def _check(s, X, p):
    A = gen.btri_dense(s.B, s.D, s.C)
    ref = oracle.dense_solve(A, s.F)
    kappa = np.linalg.cond(A, 1)
    eta = _eta(s, p)
    assert _backward_error(s, X) <= eta
    assert oracle.rel_err(X, ref) <= 1e-11 + eta * kappa


def _solve(s, p0, cuda, nrhs=None):
    import paper_0912_3678_gb300 as bt
    N, m = s.D.shape[0], s.D.shape[1]
    nr = s.F.shape[1] if nrhs is None else nrhs
    with bt.BtPlan.tuned(N, m, nr, "fp64", {"p0": p0, "pivot": 2}) as plan:
        plan.factor(*(to_dev(a, cuda) for a in (s.B, s.D, s.C)))
        X = to_host(plan.solve(to_dev(s.F, cuda)))
        plan.sync()
        p_eff = plan.levels()[0][1]
    return X, p_eff


@pytest.mark.parametrize("m", [1, 2, 4, 8, 16])
@pytest.mark.parametrize("N,p0", [(64, 4), (300, 16), (301, 1)])
def test_qr_partitions_match_dense_gepp(cuda, m, N, p0):
    s = gen.btri_nondominant(N, m, 2, seed_rep=N + 7 * m, zero_frac=0.08)
    X, p_eff = _solve(s, p0, cuda)
    _check(s, X, p0)
    assert p_eff == p0


@pytest.mark.parametrize("m,nr", [(32, 3), (3, 1), (12, 32), (16, 32)])
def test_qr_block_orders_and_many_rhs(cuda, m, nr):
    """m = 32 (the largest window), orders padded to the next power of two,
    and the full 32 right-hand sides."""
    N = 48 if m == 32 else 130
    s = gen.btri_nondominant(N, m, nr, seed_rep=31 + m, zero_frac=0.1)
    X, _ = _solve(s, 5, cuda)
    _check(s, X, 5)


def test_qr_many_singular_blocks(cuda):
    """Half the diagonal blocks exactly zero: the reduced system keeps p0 - 1
    rows (the pivoted-partition variant would split at most of them)."""
    N, m = 400, 4
    s = gen.btri_nondominant(N, m, 1, seed_rep=77, zero_frac=0.5)
    X, p_eff = _solve(s, 16, cuda)
    _check(s, X, 16)
    assert p_eff == 16


def test_qr_reduced_matrix_is_schur_complement(cuda):
    """(alpha, beta, gamma) of the QR plan equal the Schur complement of A onto
    the uniform separators, with exactly singular D_j on first local rows."""
    import paper_0912_3678_gb300 as bt
    N, m, p = 40, 2, 8
    s = gen.btri_nondominant(N, m, 1, seed_rep=5, zero_frac=0.0)
    s.D[5] = 0.0
    s.D[20] = 0.0
    with bt.BtPlan.tuned(N, m, 1, "fp64", {"p0": p, "pivot": 2}) as plan:
        plan.factor(*(to_dev(a, cuda) for a in (s.B, s.D, s.C)))
        al, be, ga = (to_host(t) for t in plan.reduced())
        plan.sync()
    A = gen.btri_dense(s.B, s.D, s.C)
    ral, rbe, rga, _, T = P.btri_reduced_blocks(A, s.F, m, N, p)
    scale = np.abs(T).max()
    K = p - 1
    assert al.shape[0] == K
    for k in range(K):
        assert np.abs(al[k] - ral[k]).max() <= 1e-12 * scale
        if k > 0:
            assert np.abs(be[k] - rbe[k]).max() <= 1e-12 * scale
        if k + 1 < K:
            assert np.abs(ga[k] - rga[k]).max() <= 1e-12 * scale


def test_qr_two_row_partitions(cuda):
    """The smallest partitions (one local row and its separator: the last
    local row's m x m step only) and a last partition of one row."""
    N, m = 59, 4
    s = gen.btri_nondominant(N, m, 2, seed_rep=8, zero_frac=0.0)
    X, p_eff = _solve(s, 30, cuda)
    _check(s, X, 30)
    assert p_eff == 30


def test_qr_refine_and_graph(cuda):
    """bt_refine on a QR plan, and a captured factor + solve replayed on new
    matrix values."""
    import paper_0912_3678_gb300 as bt
    N, m = 200, 8
    s = gen.btri_nondominant(N, m, 1, seed_rep=9, zero_frac=0.1)
    B, D, C, F = (to_dev(a, cuda) for a in (s.B, s.D, s.C, s.F))
    with bt.BtPlan.tuned(N, m, 1, "fp64", {"p0": 8, "pivot": 2}) as plan:
        plan.factor(B, D, C)
        X, it, rc, code = plan.refine(F, tol=1e-12, maxit=10)
        assert code == 0
        _check(s, to_host(X), 8)
        X2 = F.clone().zero_()
        plan.capture("factor_solve", F, X2)
        s2 = gen.btri_nondominant(N, m, 1, seed_rep=10, zero_frac=0.1)
        B.copy_(to_dev(s2.B, cuda))
        D.copy_(to_dev(s2.D, cuda))
        C.copy_(to_dev(s2.C, cuda))
        F.copy_(to_dev(s2.F, cuda))
        plan.replay()
        plan.sync()
        _check(s2, to_host(X2), 8)


def test_qr_full_size_backward_error(cuda):
    """The 16384 x 16 system of the main benchmark made non-dominant (8% of
    the diagonal blocks zero), 608 partitions: normwise backward error within
    the bound, against the oracle's partition solve and residual."""
    N, m = 16384, 16
    s = gen.btri_nondominant(N, m, 1, seed_rep=1234, zero_frac=0.08)
    X, p_eff = _solve(s, 608, cuda)
    assert p_eff == 608
    assert _backward_error(s, X) <= _eta(s, 608)


def test_qr_rejects_and_reports(cuda):
    """QR partitions factor in FP64 only; an all-zero matrix (every local
    block singular) is reported as BT_ERR_SINGULAR."""
    import paper_0912_3678_gb300 as bt
    with pytest.raises(bt.BtError):
        bt.BtPlan.tuned(64, 4, 1, "fp32_ir", {"p0": 4, "pivot": 2})
    with pytest.raises(bt.BtError):
        bt.BtPlan.tuned(64, 4, 1, "fp64", {"p0": 4, "pivot": 3})
    N, m = 64, 4
    z = np.zeros((N, m, m))
    with bt.BtPlan.tuned(N, m, 1, "fp64", {"p0": 4, "pivot": 2}) as plan:
        plan.factor(*(to_dev(z, cuda) for _ in range(3)))
        code = plan.info()[0]
    assert bt.BT_STATUS[code] == "BT_ERR_SINGULAR"
