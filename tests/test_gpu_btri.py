"""GPU parity of the block tridiagonal partition solver (bt_*) against the
oracle, element by element on the same seeded inputs.  FP64 path: normwise
relative error <= 1e-11 (the systems here have kappa <= ~10); mixed precision
with FP64 refinement: <= 1e-10."""
import numpy as np
import pytest

import gen
import oracle
from oracle import partition as P
from conftest import to_dev, to_host

pytestmark = pytest.mark.gpu

TOL64 = 1e-11
TOLIR = 1e-10


def _solve(cuda, s, p=0, prec="fp64", nrhs=None):
    import paper_0912_3678_gb300 as bt
    N, m = s.D.shape[0], s.D.shape[1]
    nr = s.F.shape[1] if nrhs is None else nrhs
    B, D, C, F = (to_dev(a, cuda) for a in (s.B, s.D, s.C, s.F))
    with bt.BtPlan(N, m, nrhs_max=nr, prec=prec, p=p) as plan:
        plan.factor(B, D, C)
        X = plan.solve(F)
        plan.sync()
        return to_host(X), plan.levels()


@pytest.mark.parametrize("m", [1, 2, 4, 8, 16, 32])
@pytest.mark.parametrize("N,nrhs", [(1, 1), (2, 2), (7, 1), (37, 3), (301, 2)])
def test_btri_fp64_matches_oracle(cuda, m, N, nrhs):
    s = gen.btri_random(N, m, nrhs, seed_rep=7 * N + m)
    X, lev = _solve(cuda, s)
    ref = oracle.btri_solve(s.B, s.D, s.C, s.F)
    assert oracle.rel_err(X, ref) <= TOL64, lev


@pytest.mark.parametrize("m", [1, 4, 16])
def test_btri_many_partitions_ragged(cuda, m):
    """Several tiles and a ragged tail: N not divisible by p, multi-level recursion."""
    N = 4099
    s = gen.btri_random(N, m, 2, seed_rep=m)
    X, lev = _solve(cuda, s)
    assert len(lev) >= 2
    ref = oracle.btri_solve(s.B, s.D, s.C, s.F)
    assert oracle.rel_err(X, ref) <= TOL64


@pytest.mark.parametrize("m", [1, 8])
def test_btri_invariant_under_p(cuda, m):
    N = 61
    s = gen.btri_random(N, m, 2, seed_rep=3)
    ref = oracle.btri_solve(s.B, s.D, s.C, s.F)
    sols = []
    for p in (1, 2, 3, 7, 30, 31):
        X, _ = _solve(cuda, s, p=p)
        assert oracle.rel_err(X, ref) <= TOL64, p
        sols.append(X)
    for X in sols[1:]:
        assert oracle.rel_err(X, sols[0]) <= 1e-13


@pytest.mark.parametrize("m,N,p", [(1, 40, 5), (2, 23, 4), (8, 30, 6), (16, 17, 3)])
def test_reduced_matrix_is_schur_complement(cuda, m, N, p):
    """The top-level reduced matrix of Eq. (redmatr) equals the Schur complement
    of the local unknowns (oracle, dense definition)."""
    import paper_0912_3678_gb300 as bt
    s = gen.btri_random(N, m, 1, seed_rep=N)
    A = gen.btri_dense(s.B, s.D, s.C)
    al, be, ga, g, T = P.btri_reduced_blocks(A, s.F, m, N, p)
    with bt.BtPlan(N, m, 1, p=p) as plan:
        plan.factor(*(to_dev(a, cuda) for a in (s.B, s.D, s.C)))
        a_, b_, g_ = (to_host(t) for t in plan.reduced())
    scale = np.abs(T).max()
    assert np.abs(a_ - al).max() <= 1e-13 * scale
    assert np.abs(b_ - be).max() <= 1e-13 * scale
    assert np.abs(g_ - ga).max() <= 1e-13 * scale


def test_scalar_n65536_p64(cuda):
    """Scalar tridiagonal n = 2^16, p = 64 partitions (the plain method)."""
    s = gen.tri_sdd(1 << 16, 1, seed_rep=0)
    sb = gen.BtriSystem(s.dl.reshape(-1, 1, 1), s.d.reshape(-1, 1, 1), s.du.reshape(-1, 1, 1), s.f, s.xstar)
    X, lev = _solve(cuda, sb, p=64)
    assert lev[0] == (1 << 16, 64)
    ref = oracle.tri_solve(s.dl, s.d, s.du, s.f)
    assert oracle.rel_err(X, ref) <= TOL64
    # and with the automatic partition count
    X2, _ = _solve(cuda, sb)
    assert oracle.rel_err(X2, ref) <= TOL64


def test_poisson_closed_form(cuda):
    """tridiag(-1,2,-1), n = 4096, f = 2: x_i = i (n+1-i); kappa ~ 6.8e6, so the
    gate is 10 kappa u (any FP64 solver's forward error bound) plus a backward
    error check."""
    n = 4096
    dl, d, du = gen.poisson(n)
    f = 2.0 * np.ones((n, 1))
    sb = gen.BtriSystem(dl.reshape(-1, 1, 1), d.reshape(-1, 1, 1), du.reshape(-1, 1, 1), f, None)
    X, _ = _solve(cuda, sb)
    i = np.arange(1, n + 1, dtype=float)
    xe = (i * (n + 1 - i))[:, None]
    lam = 2 - 2 * np.cos(np.arange(1, n + 1) * np.pi / (n + 1))
    kappa = lam.max() / lam.min()
    assert oracle.rel_err(X, xe) <= 10 * kappa * np.finfo(float).eps
    r = oracle.tri_residual(dl, d, du, X, f)
    assert np.linalg.norm(r) / (4 * np.linalg.norm(X) + np.linalg.norm(f)) <= 1e-14


def test_block_m16_n16384_full_size_fp64(cuda):
    """Block tridiagonal m = 16, N = 16384 block rows, 8 right-hand sides."""
    s = gen.btri_random(16384, 16, 8, seed_rep=0)
    X, lev = _solve(cuda, s)
    ref = oracle.btri_solve(s.B, s.D, s.C, s.F)
    assert oracle.rel_err(X, ref) <= TOL64


@pytest.mark.parametrize("prec", ["fp64", "fp32_ir"])
def test_block_m16_n16384_in_the_bench_launch_configuration(cuda, prec):
    """The block workload at full size (m = 16, N = 16384, 8 RHS) as the bench
    runs it: the autotuner's partitioning for this shape (level-0 partitions
    from the SM count, reduced system by cyclic reduction), one captured CUDA
    graph per step (factor + solve, or factor + two corrections and the
    checking residual), replayed; every entry against the oracle."""
    import paper_0912_3678_gb300 as bt
    N, m, nr = 16384, 16, 8
    s = gen.btri_random(N, m, nr, seed_rep=0)
    ref = oracle.btri_solve(s.B, s.D, s.C, s.F)
    B, D, C, F = (to_dev(a, cuda) for a in (s.B, s.D, s.C, s.F))
    with bt.BtPlan.tuned(N, m, nr, prec, {"reduced": 1}) as plan:
        plan.factor(B, D, C)
        X = plan.solve(F)
        if prec == "fp64":
            plan.capture("factor_solve", F, X)
        else:
            plan.capture("factor_refine", F, X, sweeps=2)
        X.zero_()
        plan.replay()
        plan.sync()
        if prec != "fp64":
            code, rel = bt.bt_refine_result(plan.handle, 1e-12)
            assert code == 0
        assert oracle.rel_err(to_host(X), ref) <= (TOL64 if prec == "fp64" else TOLIR)


@pytest.mark.parametrize("m,N", [(1, 5000), (4, 999), (8, 700), (16, 1024), (32, 130)])
def test_mixed_precision_refinement(cuda, m, N):
    import paper_0912_3678_gb300 as bt
    s = gen.btri_random(N, m, 3, seed_rep=11)
    ref = oracle.btri_solve(s.B, s.D, s.C, s.F)
    B, D, C, F = (to_dev(a, cuda) for a in (s.B, s.D, s.C, s.F))
    with bt.BtPlan(N, m, 3, prec="fp32_ir") as plan:
        plan.factor(B, D, C)
        X0 = to_host(plan.solve(F))
        X, it, rc, code = plan.refine(F, tol=1e-12, maxit=20)
    lo = oracle.rel_err(X0, ref)
    assert 1e-12 < lo < 1e-4            # the unrefined FP32 solve is not FP64-accurate
    assert code == 0 and 1 <= it <= 6
    assert oracle.rel_err(to_host(X), ref) <= TOLIR


@pytest.mark.parametrize("m,N", [(16, 2000), (32, 300)])
def test_bf16_tensor_core_schur_refinement(cuda, m, N):
    """BF16 operands for the Schur products (tensor cores, FP32 accumulate):
    the unrefined solve is only a few digits accurate (reported, not gated);
    FP64 refinement brings it to <= 1e-10."""
    import paper_0912_3678_gb300 as bt
    s = gen.btri_random(N, m, 2, seed_rep=13)
    ref = oracle.btri_solve(s.B, s.D, s.C, s.F)
    B, D, C, F = (to_dev(a, cuda) for a in (s.B, s.D, s.C, s.F))
    with bt.BtPlan(N, m, 2, prec="bf16_ir") as plan:
        plan.factor(B, D, C)
        lo = oracle.rel_err(to_host(plan.solve(F)), ref)
        X, it, rc, code = plan.refine(F, tol=1e-12, maxit=30)
    with bt.BtPlan(N, m, 2, prec="fp32_ir") as plan:
        plan.factor(B, D, C)
        lo32 = oracle.rel_err(to_host(plan.solve(F)), ref)
    print(f"m={m}: unrefined rel err bf16 {lo:.2e}, fp32 {lo32:.2e}; bf16 corrections {it}")
    assert lo > 10 * lo32              # the BF16 products are really in use
    assert lo < 0.5
    assert code == 0
    assert oracle.rel_err(to_host(X), ref) <= TOLIR


def test_residual_matches_oracle(cuda):
    import paper_0912_3678_gb300 as bt
    s = gen.btri_random(300, 8, 4, seed_rep=2)
    Xr = np.random.default_rng(0).standard_normal(s.F.shape)
    ref = oracle.btri_residual(s.B, s.D, s.C, Xr, s.F)
    B, D, C, F, X = (to_dev(a, cuda) for a in (s.B, s.D, s.C, s.F, Xr))
    with bt.BtPlan(300, 8, 4) as plan:
        plan.factor(B, D, C)
        R = to_host(plan.residual(F, X))
    scale = np.abs(s.F).max() + 3 * 8 * np.abs(Xr).max()
    assert np.abs(R - ref).max() <= 1e-14 * scale


def test_singular_block_is_reported(cuda):
    """A zero pivot block (host-made fault in the input) sets BT_ERR_SINGULAR."""
    import paper_0912_3678_gb300 as bt
    s = gen.btri_random(50, 4, 1, seed_rep=4)
    s.D[0] = 0.0
    s.B[1] = 0.0
    with bt.BtPlan(50, 4, 1, p=1) as plan:
        plan.factor(*(to_dev(a, cuda) for a in (s.B, s.D, s.C)))
        code, lev, part, row = plan.info()
    assert bt.BT_STATUS[code] == "BT_ERR_SINGULAR"
    assert row == 0


def test_nonfinite_input_is_reported(cuda):
    import paper_0912_3678_gb300 as bt
    s = gen.btri_random(50, 8, 1, seed_rep=4)
    s.D[10, 0, 0] = np.nan
    with bt.BtPlan(50, 8, 1) as plan:
        plan.factor(*(to_dev(a, cuda) for a in (s.B, s.D, s.C)))
        code, *_ = plan.info()
    assert bt.BT_STATUS[code] in ("BT_ERR_NONFINITE", "BT_ERR_SINGULAR")


def test_invalid_arguments(cuda):
    import paper_0912_3678_gb300 as bt
    with pytest.raises(bt.BtError):
        bt.BtPlan(10, 33)          # block order above 32
    with pytest.raises(bt.BtError):
        bt.BtPlan(10, 0)
    with pytest.raises(bt.BtError):
        bt.BtPlan(10, 4, nrhs_max=33)
    with pytest.raises(bt.BtError):
        bt.BtPlan(10, 4, p=6)      # p > (N+1)/2
    with bt.BtPlan(10, 4) as plan:
        F = to_dev(np.zeros((40, 1)), cuda)
        with pytest.raises(bt.BtError):
            plan.solve(F)          # not factored


def test_plan_on_caller_workspace_and_async_refine(cuda):
    """bt_plan_create_in builds the plan in caller memory (no allocation);
    bt_refine_async + bt_refine_result give the same answer as bt_refine."""
    import torch
    import paper_0912_3678_gb300 as bt
    N, m, nr = 900, 8, 3
    s = gen.btri_random(N, m, nr, seed_rep=21)
    ref = oracle.btri_solve(s.B, s.D, s.C, s.F)
    B, D, C, F = (to_dev(a, cuda) for a in (s.B, s.D, s.C, s.F))
    need = bt.bt_plan_workspace_size(0, N, m, nr, "fp32_ir")
    ws = torch.empty(need + 256, dtype=torch.uint8, device=cuda)
    base = ws.data_ptr() + ((-ws.data_ptr()) % 256)
    with pytest.raises(bt.BtError):
        bt.bt_plan_create_in(0, N, m, nr, "fp32_ir", base, need - 1024)
    plan = bt.bt_plan_create_in(0, N, m, nr, "fp32_ir", base, need)
    try:
        bt.bt_factor(plan, B, D, C)
        X = torch.empty_like(F)
        bt.bt_refine_async(plan, F, X, nr, 3)
        code, rel = bt.bt_refine_result(plan, 1e-12)
        assert code == 0 and rel <= 1e-12
        assert oracle.rel_err(to_host(X), ref) <= TOLIR
    finally:
        bt.bt_plan_destroy(plan)
    del ws


@pytest.mark.parametrize("m", [1, 32])
def test_largest_rhs_count(cuda, m):
    """nrhs = 32 (the maximum) with ragged sizes."""
    N = 1000 if m == 1 else 45
    s = gen.btri_random(N, m, 32, seed_rep=77)
    X, _ = _solve(cuda, s)
    assert oracle.rel_err(X, oracle.btri_solve(s.B, s.D, s.C, s.F)) <= TOL64


@pytest.mark.parametrize("prec", ["fp64", "fp32_ir"])
def test_captured_graph_replay(cuda, prec):
    """bt_plan_capture/bt_plan_replay: the graph re-reads the bound arrays."""
    import paper_0912_3678_gb300 as bt
    N, m, nr = 700, 16, 2
    s = gen.btri_random(N, m, nr, seed_rep=31)
    B, D, C, F = (to_dev(a, cuda) for a in (s.B, s.D, s.C, s.F))
    with bt.BtPlan(N, m, nr, prec=prec) as plan:
        plan.factor(B, D, C)
        X = plan.solve(F)
        if prec == "fp64":
            plan.capture("factor_solve", F, X)
        else:
            plan.capture("factor_refine", F, X, sweeps=3)
        rng = np.random.default_rng(3)
        for rep in range(2):
            s.F = rng.standard_normal(s.F.shape)
            F.copy_(to_dev(s.F, cuda))
            plan.replay()
            plan.sync()
            ref = oracle.btri_solve(s.B, s.D, s.C, s.F)
            assert oracle.rel_err(to_host(X), ref) <= (TOL64 if prec == "fp64" else TOLIR)


@pytest.mark.parametrize("m", [8, 16, 32])
@pytest.mark.parametrize("N,p", [(9, 2), (64, 3), (301, 7), (2049, 0)])
def test_cyclic_reduction_of_the_reduced_system(cuda, m, N, p):
    """Reduced system by block cyclic reduction (bt_tuning.reduced = 1)."""
    import paper_0912_3678_gb300 as bt
    s = gen.btri_random(N, m, 3, seed_rep=N + 5 * m)
    ref = oracle.btri_solve(s.B, s.D, s.C, s.F)
    B, D, C, F = (to_dev(a, cuda) for a in (s.B, s.D, s.C, s.F))
    for prec in ("fp64", "fp32_ir"):
        with bt.BtPlan.tuned(N, m, 3, prec, {"p0": p, "reduced": 1}) as plan:
            plan.factor(B, D, C)
            if prec == "fp64":
                X = plan.solve(F)
                plan.sync()
                assert oracle.rel_err(to_host(X), ref) <= TOL64
            else:
                X, it, rc, code = plan.refine(F, tol=1e-12, maxit=20)
                assert code == 0 and oracle.rel_err(to_host(X), ref) <= TOLIR
            lev = plan.levels()
            if len(lev) > 1:
                assert lev[-1][1] == 0          # the holder level of the cyclic reduction


def test_refinement_stops_on_backward_error(cuda):
    """FP32 factors of a well-conditioned system: the FP32 solve alone is not
    backward stable in FP64, so bt_refine corrects until the normwise backward
    error of x is at most 4(3m+1)u (each correction gains about kappa*u32,
    so two suffice here); with the backward-error test switched off it stops
    on the correction test, never earlier."""
    import paper_0912_3678_gb300 as bt
    from paper_0912_3678_gb300 import _lib
    N, m = 3000, 16
    s = gen.btri_random(N, m, 2, seed_rep=17)
    ref = oracle.btri_solve(s.B, s.D, s.C, s.F)
    B, D, C, F = (to_dev(a, cuda) for a in (s.B, s.D, s.C, s.F))
    eta_tol = 4 * (3 * m + 1) * 2.0 ** -53
    with bt.BtPlan(N, m, 2, prec="fp32_ir") as plan:
        plan.factor(B, D, C)
        X, it, rc, code = plan.refine(F, tol=1e-12)
        assert code == 0 and 1 <= it <= 2
        Xh = to_host(X)
        r = oracle.btri_residual(s.B, s.D, s.C, Xh, s.F)
        rows = np.abs(s.D).sum(2)
        rows[1:] += np.abs(s.B[1:]).sum(2)
        rows[:-1] += np.abs(s.C[:-1]).sum(2)
        anorm = rows.max()                             # ||A||_inf
        eta = np.abs(r).max() / (anorm * np.abs(Xh).max() + np.abs(s.F).max())
        assert eta <= 2 * eta_tol
        assert oracle.rel_err(Xh, ref) <= TOLIR
        _lib.load().bt_plan_set_backward_tol(plan.handle, 0.0)
        X2, it2, rc2, code2 = plan.refine(F, tol=1e-12)
        assert code2 == 0 and it2 >= it and rc2 <= 1e-12
        assert oracle.rel_err(to_host(X2), ref) <= TOLIR
    with bt.BtPlan(N, m, 2, prec="fp64") as plan:
        plan.factor(B, D, C)
        X, it, rc, code = plan.refine(F)
        assert code == 0 and it == 0       # the FP64 solve is already backward stable


def test_forward_tol_stops_on_the_correction_ratio(cuda):
    """bt_plan_set_forward_tol: with the backward-error test switched off
    (threshold 0) and the correction test out of reach, the refinement stops
    once rho/(1-rho) ||d_k||/||x|| (rho = ||d_k||/||d_(k-1)||, d_0 = x_0) is below
    the target; the result's error against the oracle is within 10 times the
    estimate and below the target.  The async form with the same number of
    corrections is accepted by bt_refine_result, and is not without the option."""
    import torch

    import paper_0912_3678_gb300 as bt
    N, m, nr = 4096, 16, 8
    s = gen.btri_random(N, m, nr, seed_rep=29)
    ref = oracle.btri_solve(s.B, s.D, s.C, s.F)
    B, D, C, F = (to_dev(a, cuda) for a in (s.B, s.D, s.C, s.F))
    fwd = 1e-11
    with bt.BtPlan(N, m, nr, prec="fp32_ir") as plan:
        plan.factor(B, D, C)
        bt.bt_plan_set_backward_tol(plan.handle, 0.0)
        plan.set_forward_tol(fwd)
        X, it, rc, code = plan.refine(F, tol=1e-300)
        assert code == 0 and it >= 1
        err = oracle.rel_err(to_host(X), ref)
        if it == 1:
            est = rc * rc / (1.0 - rc)       # rho = ||d_1|| / ||x_0||, ||x_0|| ~ ||x||
            assert est <= fwd and err <= 10 * est + 1e-15
        assert err <= 10 * fwd
        X2 = torch.empty_like(F)
        bt.bt_refine_async(plan.handle, F, X2, nr, it)
        code2, _ = bt.bt_refine_result(plan.handle, 1e-300)
        assert code2 == 0
        assert oracle.rel_err(to_host(X2), ref) <= 10 * fwd
        plan.set_forward_tol(0.0)
        bt.bt_refine_async(plan.handle, F, X2, nr, it)
        code3, _ = bt.bt_refine_result(plan.handle, 1e-300)
        assert bt.BT_STATUS[code3] == "BT_ERR_NOT_CONVERGED"


@pytest.mark.parametrize("m", [1, 5, 16])
def test_anorm_matches_numpy(cuda, m):
    """||A||_inf used by the stopping test (FP32 sums of truncated entries)
    agrees with the exact row-sum norm to 1e-5 relative."""
    import paper_0912_3678_gb300 as bt
    N = 777
    s = gen.btri_random(N, m, 1, seed_rep=23)
    s.D[5] *= 40.0                                  # one dominant block row
    rows = np.abs(s.D).sum(2)
    rows[1:] += np.abs(s.B[1:]).sum(2)
    rows[:-1] += np.abs(s.C[:-1]).sum(2)
    exact = rows.max()
    with bt.BtPlan(N, m, 1) as plan:
        plan.factor(*(to_dev(a, cuda) for a in (s.B, s.D, s.C)))
        got = plan.anorm()
    assert abs(got - exact) <= 1e-5 * exact


@pytest.mark.parametrize("m,N,tuning", [(1, 60000, {"p0": 2048}), (2, 30000, {}), (4, 20000, {}),
                                        (8, 3000, {}), (16, 2000, {"reduced": 1}), (16, 2000, {"reduced": 0}),
                                        (32, 400, {})])
@pytest.mark.parametrize("prec", ["fp64", "fp32_ir"])
def test_captured_step_refactors_new_matrices(cuda, m, N, tuning, prec):
    """A captured factor+solve (or factor+refine) graph runs the factorization of
    the reduced systems beside the level-0 forward substitution.  Replayed after
    the matrices AND the right-hand side are overwritten in place, it must solve
    the new system: a solve that read reduced-system factors before they were
    rewritten would return the old system's answer."""
    import paper_0912_3678_gb300 as bt
    nr = 3
    s0 = gen.btri_random(N, m, nr, seed_rep=41)
    s1 = gen.btri_random(N, m, nr, seed_rep=42)
    B, D, C, F = (to_dev(a, cuda) for a in (s0.B, s0.D, s0.C, s0.F))
    with bt.BtPlan.tuned(N, m, nr, prec, tuning) as plan:
        assert len(plan.levels()) >= 2
        plan.factor(B, D, C)
        X = plan.solve(F)
        if prec == "fp64":
            plan.capture("factor_solve", F, X)
        else:
            plan.capture("factor_refine", F, X, sweeps=3)
        for s in (s1, s0, s1):
            for dev, host in zip((B, D, C, F), (s.B, s.D, s.C, s.F)):
                dev.copy_(to_dev(host, cuda))
            X.zero_()
            plan.replay()
            plan.sync()
            ref = oracle.btri_solve(s.B, s.D, s.C, s.F)
            assert oracle.rel_err(to_host(X), ref) <= (TOL64 if prec == "fp64" else TOLIR)


@pytest.mark.parametrize("m", [2, 4])
@pytest.mark.parametrize("p0,nr", [(19456, 3), (4096, 5), (1, 6)])
def test_thread_and_lane_group_kernels(cuda, m, p0, nr):
    """Block orders 2 and 4 in FP64: a level whose partitions fill a whole wave
    of thread-per-partition CTAs (p0 = 128 per SM) runs one thread per
    partition; levels with fewer partitions run a group of m*m lanes per
    partition.  Both, mixed across levels and with right-hand-side counts that
    are not multiples of m, against the oracle."""
    import paper_0912_3678_gb300 as bt
    N = 50000 if p0 > 1 else 300
    s = gen.btri_random(N, m, nr, seed_rep=m + p0)
    ref = oracle.btri_solve(s.B, s.D, s.C, s.F)
    with bt.BtPlan.tuned(N, m, nr, "fp64", {"p0": p0}) as plan:
        plan.factor(*(to_dev(a, cuda) for a in (s.B, s.D, s.C)))
        X = to_host(plan.solve(to_dev(s.F, cuda)))
        plan.sync()
    assert oracle.rel_err(X, ref) <= TOL64


def test_singular_block_in_a_thread_per_partition_level(cuda):
    """A zero pivot block in a level run one thread per partition (m = 4,
    128 partitions per SM) sets BT_ERR_SINGULAR with its block row."""
    import paper_0912_3678_gb300 as bt
    s = gen.btri_random(50000, 4, 1, seed_rep=8)
    s.D[0] = 0.0
    with bt.BtPlan.tuned(50000, 4, 1, "fp64", {"p0": 19456}) as plan:
        plan.factor(*(to_dev(a, cuda) for a in (s.B, s.D, s.C)))
        code, lev, part, row = plan.info()
    assert bt.BT_STATUS[code] == "BT_ERR_SINGULAR"
    assert (lev, row) == (0, 0)


@pytest.mark.parametrize("m,N,tuning", [(1, 60000, {"p0": 2048}), (4, 20000, {}), (16, 2000, {"reduced": 1})])
def test_captured_step_same_with_one_or_two_streams(cuda, m, N, tuning):
    """bt_tuning.serial only changes which stream the reduced systems are
    factored on: the captured step gives bitwise the same solution both ways."""
    import paper_0912_3678_gb300 as bt
    s = gen.btri_random(N, m, 2, seed_rep=17)
    B, D, C, F = (to_dev(a, cuda) for a in (s.B, s.D, s.C, s.F))
    out = []
    for serial in (0, 1):
        with bt.BtPlan.tuned(N, m, 2, "fp64", dict(tuning, serial=serial)) as plan:
            plan.factor(B, D, C)
            X = plan.solve(F)
            plan.capture("factor_solve", F, X)
            X.zero_()
            plan.replay()
            plan.sync()
            out.append(to_host(X))
    assert np.array_equal(out[0], out[1])
    assert oracle.rel_err(out[0], oracle.btri_solve(s.B, s.D, s.C, s.F)) <= TOL64


@pytest.mark.parametrize("m,N,tuning", [(1, 60000, {"p0": 2048}), (4, 20000, {}), (8, 3000, {}),
                                        (16, 2000, {"reduced": 1}), (16, 999, {"reduced": 0}), (2, 40, {"p0": 3}),
                                        (16, 1216, {"p0": 608, "reduced": 1}), (8, 1199, {"p0": 600}),
                                        (32, 9, {"p0": 2})])
@pytest.mark.parametrize("pinned", [True, False])
def test_factor_solve_host_matches_oracle(cuda, m, N, tuning, pinned):
    """bt_factor_solve_host: host arrays in and out, block rows copied in chunks
    of partitions whose factorizations start as their rows arrive; twice on
    the same plan with different systems."""
    import torch

    import paper_0912_3678_gb300 as bt
    nr = 3
    with bt.BtPlan.tuned(N, m, nr, "fp64", tuning) as plan:
        for rep in range(2):
            s = gen.btri_random(N, m, nr, seed_rep=60 + rep)
            host = [torch.from_numpy(np.ascontiguousarray(a)) for a in (s.B, s.D, s.C, s.F)]
            if pinned:
                host = [h.pin_memory() for h in host]
            X = torch.empty(host[3].shape, dtype=torch.float64)
            X = X.pin_memory() if pinned else X.numpy()
            plan.factor_solve_host(*host, X)
            plan.sync()
            Xh = X.numpy() if pinned else X
            assert oracle.rel_err(Xh, oracle.btri_solve(s.B, s.D, s.C, s.F)) <= TOL64


@pytest.mark.parametrize("m,N", [(4, 20000), (16, 2000)])
def test_factor_refine_host_matches_oracle(cuda, m, N):
    """The refined variant of the host entry point (FP32 local factors, FP64
    corrections) reaches the refinement tolerance."""
    import torch

    import paper_0912_3678_gb300 as bt
    s = gen.btri_random(N, m, 2, seed_rep=71)
    host = [torch.from_numpy(np.ascontiguousarray(a)).pin_memory() for a in (s.B, s.D, s.C, s.F)]
    X = torch.empty(host[3].shape, dtype=torch.float64).pin_memory()
    with bt.BtPlan.tuned(N, m, 2, "fp32_ir", {}) as plan:
        plan.factor_solve_host(*host, X, sweeps=3)
        code, rel = bt.bt_refine_result(plan.handle, 1e-12)
        assert code == 0
    assert oracle.rel_err(X.numpy(), oracle.btri_solve(s.B, s.D, s.C, s.F)) <= TOLIR


def test_factor_solve_host_refuses_other_plans(cuda):
    import torch

    import paper_0912_3678_gb300 as bt
    s = gen.btri_random(100, 4, 1, seed_rep=1)
    host = [torch.from_numpy(np.ascontiguousarray(a)) for a in (s.B, s.D, s.C, s.F)]
    X = torch.empty(host[3].shape, dtype=torch.float64)
    with bt.BtPlan.tuned(100, 4, 1, "fp64", {"pivot": 1}) as plan:
        with pytest.raises(bt.BtError):
            plan.factor_solve_host(*host, X)
    with bt.BtPlan.tuned(100, 4, 1, "fp64", {}) as plan:
        with pytest.raises(bt.BtError):
            plan.factor_solve_host(*host, X, sweeps=2)      # sweeps only for refined plans


@pytest.mark.parametrize("m,N,tuning", [(16, 2000, {"reduced": 1}), (8, 3000, {}), (4, 20000, {})])
def test_captured_host_call_reads_new_host_data(cuda, m, N, tuning):
    """bt_plan_capture_host: the host-array call as one graph; replayed after the
    pinned host arrays are overwritten with another system, it solves that one."""
    import torch

    import paper_0912_3678_gb300 as bt
    nr = 2
    s0 = gen.btri_random(N, m, nr, seed_rep=80)
    host = [torch.from_numpy(np.ascontiguousarray(a)).pin_memory() for a in (s0.B, s0.D, s0.C, s0.F)]
    X = torch.empty(host[3].shape, dtype=torch.float64).pin_memory()
    with bt.BtPlan.tuned(N, m, nr, "fp64", tuning) as plan:
        plan.capture_host(*host, X)
        for rep in (81, 82):
            s = gen.btri_random(N, m, nr, seed_rep=rep)
            for h, a in zip(host, (s.B, s.D, s.C, s.F)):
                h.copy_(torch.from_numpy(np.ascontiguousarray(a)))
            X.zero_()
            plan.replay()
            plan.sync()
            assert oracle.rel_err(X.numpy(), oracle.btri_solve(s.B, s.D, s.C, s.F)) <= TOL64


def test_host_path_block_m16_n16384_full_size(cuda):
    """The end-to-end path the bench times, at the full block workload size
    (m = 16, N = 16384, 8 RHS, the autotuner's plan shape): the captured
    host-array call, replayed; every entry against the oracle."""
    import torch

    import paper_0912_3678_gb300 as bt
    N, m, nr = 16384, 16, 8
    s = gen.btri_random(N, m, nr, seed_rep=0)
    ref = oracle.btri_solve(s.B, s.D, s.C, s.F)
    host = [torch.from_numpy(np.ascontiguousarray(a)).pin_memory() for a in (s.B, s.D, s.C, s.F)]
    X = torch.empty(host[3].shape, dtype=torch.float64).pin_memory()
    with bt.BtPlan.tuned(N, m, nr, "fp64", {"p0": 608, "reduced": 1, "serial": 1}) as plan:
        plan.capture_host(*host, X)
        for _ in range(2):
            X.zero_()
            plan.replay()
            plan.sync()
            assert oracle.rel_err(X.numpy(), ref) <= TOL64
