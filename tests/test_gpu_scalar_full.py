"""The scalar throughput configurations at their full sizes, in the launch
configuration the bench times, against the oracle's Thomas solve:

* one scalar tridiagonal system of n = 2^22 (the bench's `--workload block --m 1
  --N 4194304 --nrhs 1` recipe and seed) with 38,912 level-0 partitions and
  8-row recursion partitions (`p0=38912,sub_rows=8`), every entry checked;
* the 1024 independent scalar systems of n = 2^16 of `--workload scalar_batch`,
  generated on the device as the bench does, run as one batch for each
  top-level partition length the batch tuner chooses among; every system must
  report success and a sample of 32 is checked entry by entry."""
import numpy as np
import pytest

import gen
import oracle
from conftest import to_dev, to_host

pytestmark = pytest.mark.gpu

TOL64 = 1e-11


def test_scalar_2p22_bench_partitioning_matches_oracle(cuda):
    import paper_0912_3678_gb300 as bt
    N = 1 << 22
    s = gen.btri_random(N, 1, 1, seed_rep=0)
    B, D, C, F = (to_dev(a, cuda) for a in (s.B, s.D, s.C, s.F))
    with bt.BtPlan.tuned(N, 1, 1, "fp64", {"p0": 38912, "sub_rows": 8}) as plan:
        assert plan.levels()[0] == (N, 38912)
        plan.factor(B, D, C)
        X = to_host(plan.solve(F))
        plan.sync()
    ref = oracle.tri_solve(s.B[:, 0, 0], s.D[:, 0, 0], s.C[:, 0, 0], s.F[:, 0])
    assert oracle.rel_err(X[:, 0], ref) <= TOL64


@pytest.mark.parametrize("k0", [16, 32, 64, 128])
def test_scalar_batch_1024_matches_oracle(cuda, k0):
    import torch

    import paper_0912_3678_gb300 as bt
    from paper_0912_3678_gb300 import tune
    systems = gen.batch_systems_device(gen.scalar_batch_specs(), cuda)
    torch.cuda.synchronize()
    b = bt.BtBatch(systems, ir_sweeps=4, mem_cap_bytes=80 * 2 ** 30, tuner=tune.batch_tuner(k0))
    b.run()
    code, status, _ = b.finish()
    assert code == 0
    assert len(status) == 1024 and all(st == 0 for st in status)
    rng = np.random.default_rng(k0)
    for k in sorted(rng.choice(len(systems), size=32, replace=False).tolist()):
        h = {n: systems[k][n].cpu().numpy() for n in ("B", "D", "C", "F", "X")}
        ref = oracle.tri_solve(h["B"][:, 0, 0], h["D"][:, 0, 0], h["C"][:, 0, 0], h["F"][:, 0])
        assert oracle.rel_err(h["X"][:, 0], ref) <= TOL64, k
    del b
