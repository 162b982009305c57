"""Batched solves (bt_batch_*): many uneven systems of mixed block order and
precision in one CUDA-graph launch, each checked against the oracle."""
import numpy as np
import pytest

import gen
import oracle
from conftest import to_dev, to_host

pytestmark = pytest.mark.gpu


def _systems(cuda, specs, seed=0):
    out, host = [], []
    for k, (N, m, prec, nr) in enumerate(specs):
        s = gen.btri_random(N, m, nr, seed_rep=1000 * seed + k)
        host.append(s)
        import torch
        d = {n: to_dev(getattr(s, n), cuda) for n in ("B", "D", "C", "F")}
        d["X"] = torch.full_like(d["F"], float("nan"))
        d["prec"] = prec
        out.append(d)
    return out, host


SPECS = [(1, 4, "fp64", 1), (5, 1, "fp64", 2), (700, 1, "fp32_ir", 1), (333, 2, "fp64", 3),
         (901, 4, "fp32_ir", 1), (250, 8, "fp64", 2), (64, 8, "fp32_ir", 1), (513, 16, "fp64", 1),
         (300, 16, "bf16_ir", 2), (97, 32, "fp64", 1), (40, 32, "fp32_ir", 1), (2000, 4, "fp64", 1)]


def _check(host, systems, status, specs):
    for s, d, st, (N, m, prec, nr) in zip(host, systems, status, specs):
        assert st == 0, (N, m, prec, st)
        ref = oracle.btri_solve(s.B, s.D, s.C, s.F)
        tol = 1e-11 if prec == "fp64" else 1e-10
        assert oracle.rel_err(to_host(d["X"]), ref) <= tol, (N, m, prec)


def test_batch_mixed_matches_oracle(cuda):
    import paper_0912_3678_gb300 as bt
    systems, host = _systems(cuda, SPECS)
    with bt.BtBatch(systems, ir_sweeps=5) as b:
        waves, nodes, nbytes = b.info()
        assert waves == 1 and nodes > 0
        b.run()
        code, status, rel = b.finish(tol=1e-12)
    assert code == 0
    _check(host, systems, status, SPECS)


def test_batch_waves_under_memory_cap(cuda):
    import paper_0912_3678_gb300 as bt
    systems, host = _systems(cuda, SPECS, seed=1)
    with bt.BtBatch(systems, ir_sweeps=5, mem_cap_bytes=6 << 20) as b:
        waves, _, _ = b.info()
        assert waves >= 2
        b.run()
        code, status, _ = b.finish()
    _check(host, systems, status, SPECS)


def test_batch_rerun_with_new_right_hand_sides(cuda):
    import paper_0912_3678_gb300 as bt
    specs = SPECS[:6]
    systems, host = _systems(cuda, specs, seed=2)
    with bt.BtBatch(systems, ir_sweeps=5) as b:
        b.run()
        b.finish()
        rng = np.random.default_rng(5)
        for s, d in zip(host, systems):
            s.F = rng.standard_normal(s.F.shape)
            d["F"].copy_(to_dev(s.F, d["F"].device))
        b.run()
        code, status, _ = b.finish()
    _check(host, systems, status, specs)


def test_batch_reports_a_singular_system(cuda):
    import paper_0912_3678_gb300 as bt
    specs = [(50, 4, "fp64", 1), (60, 8, "fp64", 1), (70, 4, "fp64", 1)]
    systems, host = _systems(cuda, specs, seed=3)
    host[1].D[0] = 0.0
    host[1].B[1] = 0.0
    systems[1]["D"].copy_(to_dev(host[1].D, cuda))
    systems[1]["B"].copy_(to_dev(host[1].B, cuda))
    with bt.BtBatch(systems) as b:
        b.run()
        code, status, _ = b.finish()
    assert bt.BT_STATUS[status[1]] == "BT_ERR_SINGULAR"
    assert status[0] == 0 and status[2] == 0
    for k in (0, 2):
        ref = oracle.btri_solve(host[k].B, host[k].D, host[k].C, host[k].F)
        assert oracle.rel_err(to_host(systems[k]["X"]), ref) <= 1e-11
