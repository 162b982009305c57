"""Block tridiagonal matrices with corner blocks (Sec. 2, Eqs. (parpart1),
(redmatr1) with the c couplings): the one-corner form of the paper (B_0
coupling row 0 to the last unknowns) and periodic block tridiagonal matrices
(both corners), against the oracle's dense GEPP on the dense matrix with the
corners, and the residual against the dense product."""
import numpy as np
import pytest

import gen
import oracle
from conftest import to_dev, to_host

pytestmark = pytest.mark.gpu


def _dense(B, D, C):
    N, m = D.shape[0], D.shape[1]
    A = gen.btri_dense(B, D, C)
    A[:m, (N - 1) * m:] += B[0]
    A[(N - 1) * m:, :m] += C[N - 1]
    return A


def _system(N, m, nr, seed, corners=2, nondominant=False):
    s = (gen.btri_nondominant(N, m, nr, seed_rep=seed, zero_frac=0.0) if nondominant
         else gen.btri_random(N, m, nr, seed_rep=seed))
    rng = np.random.default_rng(seed)
    B, D, C = s.B.copy(), s.D.copy(), s.C.copy()
    B[0] = rng.standard_normal((m, m)) / np.sqrt(m)
    C[N - 1] = rng.standard_normal((m, m)) / np.sqrt(m) if corners == 2 else 0.0
    A = _dense(B, D, C)
    F = A @ s.Xstar
    return B, D, C, F, A


@pytest.mark.parametrize("m", [1, 2, 3, 4, 8, 16, 32])
@pytest.mark.parametrize("N,p,corners", [(40, 4, 2), (129, 8, 2), (64, 0, 1), (4, 1, 2)])
def test_corner_matrix_matches_dense_gepp(cuda, m, N, p, corners):
    import paper_0912_3678_gb300 as bt
    nr = 3
    B, D, C, F, A = _system(N, m, nr, seed=N + m, corners=corners)
    ref = oracle.dense_solve(A, F)
    with bt.PbtPlan(N, m, nr, p=p) as plan:
        plan.factor(*(to_dev(a, cuda) for a in (B, D, C)))
        Fd = to_dev(F, cuda)
        X = plan.solve(Fd)
        R = to_host(plan.residual(Fd, X))
        plan.sync()
    X = to_host(X)
    kappa = np.linalg.cond(A, 1)
    assert oracle.rel_err(X, ref) <= 1e-13 * kappa
    Rref = F - A @ X
    assert np.abs(R - Rref).max() <= 1e-13 * (np.abs(A).sum(1).max() * np.abs(X).max() + np.abs(F).max())


def test_periodic_nondominant_and_many_rhs(cuda):
    """Not diagonally dominant blocks, 32 right-hand sides, m = 16 (the inner
    plan solves the 2m = 32 coupling columns in two parts)."""
    import paper_0912_3678_gb300 as bt
    N, m, nr = 200, 16, 32
    B, D, C, F, A = _system(N, m, nr, seed=5, corners=2, nondominant=True)
    ref = oracle.dense_solve(A, F)
    with bt.PbtPlan(N, m, nr, p=8) as plan:
        plan.factor(*(to_dev(a, cuda) for a in (B, D, C)))
        X = to_host(plan.solve(to_dev(F, cuda)))
        plan.sync()
    assert oracle.rel_err(X, ref) <= 1e-12 * np.linalg.cond(A, 1)


def test_corner_plan_reports_singular_end_block(cuda):
    """A matrix whose end rows are zero: the 2m x 2m Schur complement onto the
    end separators is singular and is reported."""
    import paper_0912_3678_gb300 as bt
    N, m = 20, 4
    B, D, C, F, A = _system(N, m, 1, seed=9)
    for X in (B, D, C):
        X[0] = 0.0
    with bt.PbtPlan(N, m, 1) as plan:
        plan.factor(*(to_dev(a, cuda) for a in (B, D, C)))
        with pytest.raises(bt.BtError):
            plan.sync()
    with pytest.raises(bt.BtError):
        bt.PbtPlan(3, 4, 1)
