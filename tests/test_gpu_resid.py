"""The refinement residual r = f - A x as refined plans form it, entry by entry
against the oracle's FP64 residual (bt_refine_residual / abd_refine_residual):
the tensor-core residual (plans of block order 16 without the warp kernels --
here BF16 plans -- and at most 8 right-hand sides: error-free split into 8-bit
digit planes, Ozaki-Ogita-Oishi-Rump 2012) and the double-float residuals
(compensated dot products, Ogita-Rump-Oishi 2005): from the split copy the
order-16 warp factorization leaves, and from the FP64 matrix for the other
shapes.  All return r rounded to FP32 precision."""
import numpy as np
import pytest

import gen
import oracle
from conftest import to_dev, to_host

pytestmark = pytest.mark.gpu

U = 2.0 ** -53


def _abs_product(B, D, C, X):
    """(|A| |X|) row by row for the block tridiagonal A."""
    N, m = D.shape[0], D.shape[1]
    Xb = np.abs(X).reshape(N, m, -1)
    out = np.einsum("jik,jkc->jic", np.abs(D), Xb)
    out[1:] += np.einsum("jik,jkc->jic", np.abs(B[1:]), Xb[:-1])
    out[:-1] += np.einsum("jik,jkc->jic", np.abs(C[:-1]), Xb[1:])
    return out.reshape(N * m, -1)


def _row_bound(B, D, C, X):
    """max_k |a_ik| over row i of [B_j D_j C_j] times 3m max |x| over the
    window of block row j (the scale of the digit-plane split)."""
    N, m = D.shape[0], D.shape[1]
    amax = np.maximum(np.abs(D).max(2), 0.0)
    amax[1:] = np.maximum(amax[1:], np.abs(B[1:]).max(2))
    amax[:-1] = np.maximum(amax[:-1], np.abs(C[:-1]).max(2))
    Xb = np.abs(X).reshape(N, m, -1).max(1)            # [N][nr]
    win = Xb.copy()
    win[1:] = np.maximum(win[1:], Xb[:-1])
    win[:-1] = np.maximum(win[:-1], Xb[1:])
    return (amax[:, :, None] * 3 * m * win[:, None, :]).reshape(N * m, -1)


def _check(R, ref, bound):
    err = np.abs(R - ref)
    assert np.all(err <= bound + 2.0 ** -23 * np.abs(ref)), float((err - bound - 2.0 ** -23 * np.abs(ref)).max())


def _plan_residual(s, X, prec, nr, cuda, tuning=None):
    import paper_0912_3678_gb300 as bt
    N, m = s.D.shape[0], s.D.shape[1]
    with bt.BtPlan.tuned(N, m, nr, prec, tuning or {}) as plan:
        plan.factor(*(to_dev(a, cuda) for a in (s.B, s.D, s.C)))
        R = to_host(plan.refine_residual(to_dev(s.F, cuda), to_dev(X, cuda)))
        plan.sync()
    return R


@pytest.mark.parametrize("nr", [1, 3, 8])
@pytest.mark.parametrize("N", [7, 300])
def test_tensor_core_residual_matches_oracle(cuda, N, nr):
    """m = 16: an arbitrary X (|r| of the order of |A||x|) and a near-solution
    X (|r| near the rounding level), per entry within 2^-45 of the split's
    scale plus the FP32 rounding of r."""
    s = gen.btri_random(N, 16, nr, seed_rep=40 + N + nr)
    rng = np.random.default_rng(N * nr)
    for X in (rng.standard_normal(s.F.shape), s.Xstar * (1 + 1e-9 * rng.standard_normal(s.F.shape))):
        ref = oracle.btri_residual(s.B, s.D, s.C, X, s.F)
        R = _plan_residual(s, X, "bf16_ir", nr, cuda)
        _check(R, ref, 2.0 ** -45 * (_row_bound(s.B, s.D, s.C, X) + np.abs(s.F)))


def test_tensor_core_residual_scales(cuda):
    """Entries far from 1 (A scaled by 2^40, X by 2^-30, rows of widely
    different size), a zero block row of X and zero right-hand sides."""
    N, m, nr = 64, 16, 4
    s = gen.btri_random(N, m, nr, seed_rep=77)
    rng = np.random.default_rng(5)
    scale = 2.0 ** rng.integers(-20, 21, size=(N, m, 1))
    B, D, C = (a * scale * 2.0 ** 40 for a in (s.B, s.D, s.C))
    X = rng.standard_normal(s.F.shape) * 2.0 ** -30
    X[16 * 10:16 * 11] = 0.0
    t = gen.BtriSystem(B, D, C, s.F * 2.0 ** 10, s.Xstar)
    ref = oracle.btri_residual(B, D, C, X, t.F)
    R = _plan_residual(t, X, "bf16_ir", nr, cuda)
    _check(R, ref, 2.0 ** -45 * (_row_bound(B, D, C, X) + np.abs(t.F)))


@pytest.mark.parametrize("m,nr", [(16, 8), (16, 1), (16, 12), (8, 4), (32, 2), (4, 3)])
def test_double_float_residual_matches_oracle(cuda, m, nr):
    """The double-float kernels (FP32 plans: m = 16 from the warp
    factorization's split copy, the other orders from the FP64 matrix): per
    entry within 2^-43 of sum_k |a_ik||x_k| + |f_i| plus the FP32 rounding."""
    N = 200
    s = gen.btri_random(N, m, nr, seed_rep=90 + m)
    X = np.random.default_rng(m).standard_normal(s.F.shape)
    ref = oracle.btri_residual(s.B, s.D, s.C, X, s.F)
    R = _plan_residual(s, X, "fp32_ir", nr, cuda)
    _check(R, ref, 2.0 ** -43 * (_abs_product(s.B, s.D, s.C, X) + np.abs(s.F)))


def test_fp64_plan_residual_is_fp64(cuda):
    """A BT_FP64 plan's refinement residual is the FP64 one (no FP32 rounding)."""
    N, m, nr = 100, 16, 2
    s = gen.btri_random(N, m, nr, seed_rep=3)
    X = np.random.default_rng(1).standard_normal(s.F.shape)
    ref = oracle.btri_residual(s.B, s.D, s.C, X, s.F)
    R = _plan_residual(s, X, "fp64", nr, cuda)
    assert np.abs(R - ref).max() <= 64 * U * (_abs_product(s.B, s.D, s.C, X) + np.abs(s.F)).max()


def test_babd_double_float_residual_matches_oracle(cuda):
    import paper_0912_3678_gb300 as bt
    b = gen.babd_bvp(4096, 8, 3)
    Y = np.random.default_rng(2).standard_normal(b.RHS.shape)
    ref = oracle.babd_residual(b.S, b.R, b.B0, b.B1, Y, b.RHS)
    with bt.AbdPlan.tuned(4096, 8, 3, "fp32_ir") as plan:
        plan.factor(*(to_dev(a, cuda) for a in (b.S, b.R, b.B0, b.B1)))
        R = to_host(plan.refine_residual(to_dev(b.RHS, cuda), to_dev(Y, cuda)))
        plan.sync()
    N1, m = b.S.shape[0] + 1, 8
    Yb = np.abs(Y).reshape(N1, m, -1)
    absp = np.zeros_like(Yb)
    absp[0] = np.abs(b.B0) @ Yb[0] + np.abs(b.B1) @ Yb[-1]
    absp[1:] = np.einsum("jik,jkc->jic", np.abs(b.S), Yb[:-1]) + np.einsum("jik,jkc->jic", np.abs(b.R), Yb[1:])
    bound = 2.0 ** -43 * (absp.reshape(N1 * m, -1) + np.abs(b.RHS))
    _check(R, ref, bound)
