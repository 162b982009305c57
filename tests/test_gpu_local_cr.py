"""Local cyclic reduction (bt_tuning.local = L, the cyclic-reduction
factorization of Sec. 2): partitions of 2^L block rows reduced by odd-even
steps that never eliminate a separator (the rows at multiples of 2^L), then
the reduced system on the separators by FP64 cyclic reduction.  Checked
against the oracle element by element, against the Schur complement onto the
separators, and for invariance under L."""
import numpy as np
import pytest

import gen
import oracle
from oracle import partition as P
from conftest import to_dev, to_host

pytestmark = pytest.mark.gpu

TOL64 = 1e-11
TOLIR = 1e-10


def _plan(bt, N, m, nr, prec, L):
    return bt.BtPlan.tuned(N, m, nr, prec, {"local": L})


@pytest.mark.parametrize("m", [8, 16, 32])
@pytest.mark.parametrize("N,nrhs", [(1, 1), (2, 2), (7, 1), (37, 3), (301, 8)])
@pytest.mark.parametrize("L", [1, 3, 6])
def test_local_cr_fp64_matches_oracle(cuda, m, N, nrhs, L):
    import paper_0912_3678_gb300 as bt
    s = gen.btri_random(N, m, nrhs, seed_rep=11 * N + m + L)
    ref = oracle.btri_solve(s.B, s.D, s.C, s.F)
    with _plan(bt, N, m, nrhs, "fp64", L) as plan:
        plan.factor(*(to_dev(a, cuda) for a in (s.B, s.D, s.C)))
        X = to_host(plan.solve(to_dev(s.F, cuda)))
        plan.sync()
    assert oracle.rel_err(X, ref) <= TOL64


@pytest.mark.parametrize("m", [8, 16, 32])
@pytest.mark.parametrize("N,nrhs", [(2, 1), (37, 3), (1000, 8)])
@pytest.mark.parametrize("L", [1, 2, 5])
def test_local_cr_fp32_refined_matches_oracle(cuda, m, N, nrhs, L):
    """FP32 local steps (the reduced system stays FP64), FP64 refinement."""
    import paper_0912_3678_gb300 as bt
    s = gen.btri_random(N, m, nrhs, seed_rep=13 * N + m + L)
    ref = oracle.btri_solve(s.B, s.D, s.C, s.F)
    with _plan(bt, N, m, nrhs, "fp32_ir", L) as plan:
        plan.factor(*(to_dev(a, cuda) for a in (s.B, s.D, s.C)))
        X, it, rc, code = plan.refine(to_dev(s.F, cuda), tol=1e-12, maxit=20)
    assert code == 0
    assert oracle.rel_err(to_host(X), ref) <= TOLIR


@pytest.mark.parametrize("N,L", [(37, 2), (64, 3), (100, 1)])
def test_local_cr_reduced_is_schur_complement(cuda, N, L):
    """After L steps the FP64 system left equals the Schur complement of A onto
    the separators 0, 2^L, 2*2^L, ... (dense definition in the oracle)."""
    import paper_0912_3678_gb300 as bt
    m = 8
    s = gen.btri_random(N, m, 1, seed_rep=N + L)
    A = gen.btri_dense(s.B, s.D, s.C)
    seps = list(range(0, N, 2 ** L))
    local = [(a + 1, b) for a, b in zip(seps, seps[1:] + [N])]
    T, _ = P.schur_reduced(A, s.F, m, local, seps)
    K = len(seps)
    with _plan(bt, N, m, 1, "fp64", L) as plan:
        plan.factor(*(to_dev(a, cuda) for a in (s.B, s.D, s.C)))
        al, be, ga = (to_host(t) for t in plan.reduced())
    assert al.shape[0] == K
    scale = np.abs(T).max()
    for k in range(K):
        blk = T[k * m:(k + 1) * m]
        assert np.abs(al[k] - blk[:, k * m:(k + 1) * m]).max() <= 1e-12 * scale
        if k > 0:
            assert np.abs(be[k] - blk[:, (k - 1) * m:k * m]).max() <= 1e-12 * scale
        if k + 1 < K:
            assert np.abs(ga[k] - blk[:, (k + 1) * m:(k + 2) * m]).max() <= 1e-12 * scale
    # nothing couples separators that are not neighbours
    for k in range(K):
        for j in range(K):
            if abs(j - k) > 1:
                assert np.abs(T[k * m:(k + 1) * m, j * m:(j + 1) * m]).max() <= 1e-12 * scale


def test_local_cr_invariant_under_L(cuda):
    """The solution does not depend on the partition length 2^L."""
    import paper_0912_3678_gb300 as bt
    N, m = 777, 16
    s = gen.btri_random(N, m, 2, seed_rep=5)
    ref = oracle.btri_solve(s.B, s.D, s.C, s.F)
    B, D, C, F = (to_dev(a, cuda) for a in (s.B, s.D, s.C, s.F))
    sols = []
    for L in (1, 2, 4, 7, 10, 20):
        with _plan(bt, N, m, 2, "fp64", L) as plan:
            plan.factor(B, D, C)
            sols.append(to_host(plan.solve(F)))
            plan.sync()
    for X in sols:
        assert oracle.rel_err(X, ref) <= TOL64
        assert oracle.rel_err(X, sols[0]) <= TOL64


def test_local_cr_general_block_order_and_graph(cuda):
    """A block order embedded in the next supported one (m = 12 -> 16), FP32
    local steps, refinement captured in a CUDA graph and replayed."""
    import paper_0912_3678_gb300 as bt
    N, m, nr = 500, 12, 3
    s = gen.btri_random(N, m, nr, seed_rep=9)
    ref = oracle.btri_solve(s.B, s.D, s.C, s.F)
    B, D, C, F = (to_dev(a, cuda) for a in (s.B, s.D, s.C, s.F))
    with _plan(bt, N, m, nr, "fp32_ir", 4) as plan:
        plan.factor(B, D, C)
        X, it, rc, code = plan.refine(F, tol=1e-12, maxit=20)
        assert code == 0 and oracle.rel_err(to_host(X), ref) <= TOLIR
        X2 = X.clone().zero_()
        plan.capture("factor_refine", F, X2, sweeps=max(it, 1) + 1)
        plan.replay()
        code2, rel = bt.bt_refine_result(plan.handle, 1e-12)
        assert code2 == 0
        assert oracle.rel_err(to_host(X2), ref) <= TOLIR


def test_local_cr_reports_a_singular_block(cuda):
    """A zero row block (host-made fault in the input) on a row eliminated by
    the first step sets BT_ERR_SINGULAR with its block row."""
    import paper_0912_3678_gb300 as bt
    N, m = 64, 8
    s = gen.btri_random(N, m, 1, seed_rep=3)
    s.D[5] = 0.0
    s.B[5] = 0.0
    s.C[5] = 0.0
    with _plan(bt, N, m, 1, "fp64", 3) as plan:
        plan.factor(*(to_dev(a, cuda) for a in (s.B, s.D, s.C)))
        code, lev, part, row = plan.info()
    assert bt.BT_STATUS[code] == "BT_ERR_SINGULAR"
    assert row == 5


def test_local_cr_needs_blocks_of_order_8(cuda):
    import paper_0912_3678_gb300 as bt
    with pytest.raises(bt.BtError):
        bt.BtPlan.tuned(100, 4, 1, "fp64", {"local": 2})
