"""bt_solve_noalloc: the solve for callers that may not allocate device
memory (a host application that owns all device memory through its own pool,
or a hot loop that cannot accept cudaMalloc's implicit synchronisation).  It
must give the FP64 oracle's answer and the same answer as the plan-based
entry points, on consecutive calls that share its static scratch array, and
refuse problems larger than that array.  This file sorts last so that a run
stopping at the first failure has already run every other test."""
import ctypes

import numpy as np
import pytest

import gen
import oracle
from conftest import to_dev, to_host

pytestmark = pytest.mark.gpu

TOL64 = 1e-11   # the FP64 parity tolerance of the other GPU tests


def _plan_solve(bt, s, cuda):
    N, m = s.D.shape[0], s.D.shape[1]
    with bt.BtPlan(N, m, nrhs_max=s.F.shape[1]) as plan:
        plan.factor(*(to_dev(a, cuda) for a in (s.B, s.D, s.C)))
        X = plan.solve(to_dev(s.F, cuda))
        plan.sync()
        return to_host(X)


def _noalloc_solve(lib, s, cuda):
    import torch
    N, m = s.D.shape[0], s.D.shape[1]
    nr = s.F.shape[1]
    B, D, C, F = (to_dev(a, cuda) for a in (s.B, s.D, s.C, s.F))
    X = torch.full_like(F, float("nan"))
    req = ctypes.c_int64(0)
    code = lib.bt_solve_noalloc(N, m, B.data_ptr(), D.data_ptr(), C.data_ptr(), F.data_ptr(), X.data_ptr(),
                                nr, torch.cuda.current_stream().cuda_stream, ctypes.byref(req))
    return code, req.value, to_host(X)


def test_noalloc_matches_plan_on_consecutive_calls(cuda):
    import paper_0912_3678_gb300 as bt
    from paper_0912_3678_gb300 import _lib
    lib = _lib.load()
    cases = [gen.btri_random(300, 8, 2, seed_rep=41), gen.btri_random(123, 16, 3, seed_rep=42),
             gen.btri_random(300, 8, 2, seed_rep=43)]
    for s in cases:                        # consecutive calls share (and reuse) the scratch
        code, req, X = _noalloc_solve(lib, s, cuda)
        assert code == 0, bt.bt_status_string(code)
        assert 0 < req <= bt.BT_NOALLOC_SCRATCH_BYTES
        assert oracle.rel_err(X, oracle.btri_solve(s.B, s.D, s.C, s.F)) <= TOL64
        ref = _plan_solve(bt, s, cuda)
        err = np.linalg.norm(X - ref) / np.linalg.norm(ref)
        assert err <= TOL64


def test_noalloc_scalar_and_singular_status(cuda):
    import paper_0912_3678_gb300 as bt
    from paper_0912_3678_gb300 import _lib
    lib = _lib.load()
    t = gen.tri_sdd(20000, 1, seed_rep=5)
    s = gen.BtriSystem(t.dl.reshape(-1, 1, 1), t.d.reshape(-1, 1, 1), t.du.reshape(-1, 1, 1), t.f, t.xstar)
    code, req, X = _noalloc_solve(lib, s, cuda)
    assert code == 0
    assert oracle.rel_err(X, oracle.tri_solve(t.dl, t.d, t.du, t.f)) <= TOL64
    ref = _plan_solve(bt, s, cuda)
    assert np.linalg.norm(X - ref) / np.linalg.norm(ref) <= TOL64
    bad = gen.btri_random(40, 4, 1, seed_rep=6)
    bad.D[0] = 0.0
    bad.B[1] = 0.0
    code, _, _ = _noalloc_solve(lib, bad, cuda)
    assert bt.BT_STATUS[code] == "BT_ERR_SINGULAR"
    # a clean call right after a failed one starts from a cleared status word
    code, _, X = _noalloc_solve(lib, s, cuda)
    assert code == 0


def test_noalloc_rejects_problems_beyond_the_scratch(cuda):
    import paper_0912_3678_gb300 as bt
    from paper_0912_3678_gb300 import _lib
    import torch
    lib = _lib.load()
    req = ctypes.c_int64(0)
    # real (small) device buffers: the call must refuse on size alone, but if
    # that check ever moved behind a launch, the kernels would read valid memory
    a = torch.zeros(32 * 32, dtype=torch.float64, device=cuda)
    f = torch.zeros(32, dtype=torch.float64, device=cuda)
    x = torch.full_like(f, 7.0)
    code = lib.bt_solve_noalloc(100000, 32, a.data_ptr(), a.data_ptr(), a.data_ptr(), f.data_ptr(), x.data_ptr(), 1,
                                torch.cuda.current_stream().cuda_stream, ctypes.byref(req))
    torch.cuda.synchronize()
    assert bt.BT_STATUS[code] == "BT_ERR_INVALID"
    assert req.value > bt.BT_NOALLOC_SCRATCH_BYTES
    assert bool((x == 7.0).all())          # nothing was written
