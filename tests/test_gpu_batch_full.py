"""The full-size batch configuration: 4096 uneven independent block
tridiagonal systems (n log-uniform in [1e3, 1e6], m from {1, 4, 8, 16, 32},
half FP64 and half BF16 + refinement), run as one batch under an 80 GB memory
cap, with a sample of systems checked against the oracle's block Thomas
solve.  Every system must report success."""
import numpy as np
import pytest

import gen
import oracle

pytestmark = pytest.mark.gpu


def test_full_batch_sample_matches_oracle(cuda):
    import torch

    import paper_0912_3678_gb300 as bt
    from paper_0912_3678_gb300 import tune
    specs = gen.batch_specs(4096, nmax=1e6)
    systems = gen.batch_systems_device(specs, cuda)
    torch.cuda.synchronize()
    b = bt.BtBatch(systems, ir_sweeps=4, mem_cap_bytes=80 * 2 ** 30, tuner=tune.batch_tuner(32))
    b.run()
    code, status, rel = b.finish()
    assert code == 0
    assert len(status) == 4096 and all(s == 0 for s in status)
    rng = np.random.default_rng(7)
    sample = sorted(rng.choice(len(systems), size=40, replace=False).tolist())
    # every block order and both precisions among the checked systems
    picked = {(systems[k]["D"].shape[1], systems[k]["prec"]) for k in sample}
    for m in (1, 4, 8, 16, 32):
        for prec in ("fp64", "bf16_ir"):
            if (m, prec) not in picked:
                k = next(i for i, sd in enumerate(systems) if sd["D"].shape[1] == m and sd["prec"] == prec)
                sample.append(k)
    for k in sample:
        sd = systems[k]
        h = {n: sd[n].cpu().numpy() for n in ("B", "D", "C", "F", "X")}
        ref = oracle.btri_solve(h["B"], h["D"], h["C"], h["F"])
        tol = 1e-11 if sd["prec"] == "fp64" else 1e-10
        assert oracle.rel_err(h["X"], ref) <= tol, (k, sd["prec"], h["D"].shape)
    del b
