"""Autotuner: cache keys and persistence (CPU), and on the GPU that a tuned
plan still solves to FP64 accuracy."""
import json

import pytest

from paper_0912_3678_gb300 import tune


def test_cache_roundtrip(tmp_path):
    t = tune.Tuner(str(tmp_path / "c.json"), sm_count=152)
    assert t(16, 16384, "fp64") == tune.default_tuning(16, 16384)
    k = t.key(16, 16384, "fp64")
    assert k == "sm152:m16:fp64:n2^14:r1"
    t.cache[k] = {"tuning": {"p0": 512, "ctas_per_sm": 0, "sub_rows": 3, "top_rows": 4}, "ms": 1.0, "trials": 3}
    t.save()
    t2 = tune.Tuner(str(tmp_path / "c.json"), sm_count=152)
    assert t2(16, 16000, "fp64")["p0"] == 512          # same log2 bucket
    assert t2(16, 4000, "fp64")["p0"] == 0             # other bucket: defaults
    assert json.load(open(tmp_path / "c.json"))[k]["trials"] == 3


def test_candidates_respect_partition_bounds():
    t = tune.Tuner("/nonexistent/x.json", sm_count=152)
    for m, N in [(16, 100), (1, 50), (32, 7)]:
        for c in t.candidates_k0(m, N):
            assert 1 <= c["p0"] <= max(1, (N + 1) // 2)


@pytest.mark.gpu
def test_tuned_plan_solves(cuda, tmp_path):
    import gen
    import oracle
    from conftest import to_dev, to_host
    import paper_0912_3678_gb300 as bt
    t = tune.Tuner(str(tmp_path / "c.json"))
    best = t.tune(8, 3000, "fp64", reps=2)
    s = gen.btri_random(3000, 8, 1, seed_rep=9)
    with bt.BtPlan.tuned(3000, 8, 1, "fp64", best) as plan:
        plan.factor(*(to_dev(a, cuda) for a in (s.B, s.D, s.C)))
        X = to_host(plan.solve(to_dev(s.F, cuda)))
    assert oracle.rel_err(X, oracle.btri_solve(s.B, s.D, s.C, s.F)) <= 1e-11
