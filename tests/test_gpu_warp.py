"""GPU parity of the warp-per-partition FP32 local factorization (blocks of
order 16, used by the refined paths): the reduced matrix it leaves against
the Schur complement of the local unknowns (oracle, dense definition) within
FP32 rounding, the unrefined FP32 solve within FP32 accuracy, and the refined
solution against the FP64 oracle (<= 1e-10), over partition counts with
ragged tails, two-row partitions and a single partition; the slab-by-slab
(phased) factorization of the host-array entry point; a singular pivot block;
inputs off a 16-byte boundary (served by the CTA kernel instead)."""
import numpy as np
import pytest

import gen
import oracle
from oracle import partition as P
from conftest import to_dev, to_host

pytestmark = pytest.mark.gpu

TOLIR = 1e-10
M = 16


@pytest.mark.parametrize("N,p", [(17, 3), (40, 2), (64, 7), (100, 12), (127, 64)])
def test_fp32_reduced_matrix_is_schur_complement(cuda, N, p):
    """alpha, beta, gamma of Eq. (redmatr) from FP32 local factors equal the
    dense Schur complement up to FP32 rounding (and are not FP64-exact)."""
    import paper_0912_3678_gb300 as bt
    s = gen.btri_random(N, M, 1, seed_rep=N + 1)
    A = gen.btri_dense(s.B, s.D, s.C)
    al, be, ga, g, T = P.btri_reduced_blocks(A, s.F, M, N, p)
    with bt.BtPlan(N, M, 1, prec="fp32_ir", p=p) as plan:
        plan.factor(*(to_dev(a, cuda) for a in (s.B, s.D, s.C)))
        a_, b_, g_ = (to_host(t) for t in plan.reduced())
    scale = np.abs(T).max()
    err = max(np.abs(a_ - al).max(), np.abs(b_ - be).max(), np.abs(g_ - ga).max())
    assert err <= 2e-5 * scale
    assert err > 1e-13 * scale            # the local factors really are FP32


@pytest.mark.parametrize("N,p,nr", [(1, 1, 1), (2, 1, 2), (9, 1, 3), (33, 2, 1), (300, 150, 2),
                                    (1001, 37, 8), (4099, 0, 5), (700, 0, 12), (300, 20, 32),
                                    (16384, 608, 8)])
def test_fp32_solve_and_refinement(cuda, N, p, nr):
    import paper_0912_3678_gb300 as bt
    s = gen.btri_random(N, M, nr, seed_rep=3 * N + nr)
    ref = oracle.btri_solve(s.B, s.D, s.C, s.F)
    B, D, C, F = (to_dev(a, cuda) for a in (s.B, s.D, s.C, s.F))
    with bt.BtPlan(N, M, nr, prec="fp32_ir", p=p) as plan:
        plan.factor(B, D, C)
        lo = oracle.rel_err(to_host(plan.solve(F)), ref)
        X, it, rc, code = plan.refine(F, tol=1e-12, maxit=20)
        plan.sync()
    assert lo < 1e-4
    if N > 1:
        assert lo > 1e-12                 # FP32 factors, not FP64
    assert code == 0 and it <= 4
    assert oracle.rel_err(to_host(X), ref) <= TOLIR


@pytest.mark.parametrize("N,tuning", [(2000, {}), (1217, {"p0": 608}), (607, {"p0": 200}), (5000, {"p0": 1216})])
def test_fp32_phased_host_path(cuda, N, tuning):
    """bt_factor_solve_host factors level 0 in four row slabs, each launch
    resuming from the stored Y, Zc and the running W, Pf; with partitions of
    two or three rows some slabs are empty."""
    import torch

    import paper_0912_3678_gb300 as bt
    s = gen.btri_random(N, M, 2, seed_rep=N)
    host = [torch.from_numpy(np.ascontiguousarray(a)).pin_memory() for a in (s.B, s.D, s.C, s.F)]
    X = torch.empty(host[3].shape, dtype=torch.float64).pin_memory()
    with bt.BtPlan.tuned(N, M, 2, "fp32_ir", tuning) as plan:
        plan.factor_solve_host(*host, X, sweeps=3)
        code, rel = bt.bt_refine_result(plan.handle, 1e-12)
        assert code == 0
    assert oracle.rel_err(X.numpy(), oracle.btri_solve(s.B, s.D, s.C, s.F)) <= TOLIR


def test_fp32_singular_block_is_reported(cuda):
    """D_5 = 0 with B_5 = 0 makes the pivot block D'_5 exactly zero: the warp
    kernel reports BT_ERR_SINGULAR at block row 5."""
    import paper_0912_3678_gb300 as bt
    s = gen.btri_random(50, M, 1, seed_rep=4)
    s.D[5] = 0.0
    s.B[5] = 0.0
    with bt.BtPlan(50, M, 1, prec="fp32_ir", p=1) as plan:
        plan.factor(*(to_dev(a, cuda) for a in (s.B, s.D, s.C)))
        code, lev, part, row = plan.info()
    assert bt.BT_STATUS[code] == "BT_ERR_SINGULAR"
    assert (lev, row) == (0, 5)


def test_fp32_inputs_off_16_byte_boundary(cuda):
    """Blocks that start 8 bytes past a 16-byte boundary cannot be staged with
    16-byte copies; the plan then uses the CTA kernel, with the same result."""
    import torch

    import paper_0912_3678_gb300 as bt
    N, nr = 700, 2
    s = gen.btri_random(N, M, nr, seed_rep=19)
    ref = oracle.btri_solve(s.B, s.D, s.C, s.F)
    views = []
    for a in (s.B, s.D, s.C):
        big = torch.zeros(a.size + 1, dtype=torch.float64, device=cuda)
        v = big[1:].view(a.shape)
        v.copy_(to_dev(a, cuda))
        assert v.data_ptr() % 16 == 8
        views.append(v)
    F = to_dev(s.F, cuda)
    with bt.BtPlan(N, M, nr, prec="fp32_ir") as plan:
        plan.factor(*views)
        X, it, rc, code = plan.refine(F, tol=1e-12, maxit=20)
    assert code == 0
    assert oracle.rel_err(to_host(X), ref) <= TOLIR
