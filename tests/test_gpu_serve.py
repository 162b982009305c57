"""Serving (paper_0912_3678_gb300.serve): each request's result is the same
alone and in the mix, matches the oracle, memory admission holds the cap,
and repeated problems reuse their factorization."""
import numpy as np
import pytest

import gen
import oracle
from conftest import to_host

pytestmark = pytest.mark.gpu


def _requests(count=12, seed=0, precs=("fp64", "fp32_ir")):
    from paper_0912_3678_gb300 import serve
    rng = np.random.default_rng(seed)
    specs = {}
    out = []
    for k in range(count):
        if specs and rng.uniform() < 0.3:
            pid = int(rng.choice(list(specs)))
            m, N = specs[pid][1], specs[pid][2]
        else:
            pid = len(specs)
            m = int(rng.choice([4, 8, 16]))
            N = int(rng.integers(300, 3000))
            p = gen.bvp_problem(m, 1, seed_rep=100 + pid)
            specs[pid] = (serve.BvpSpec(p.Smat, p.K, p.B0, p.B1), m, N)
        nrhs = int(rng.integers(1, 9))
        V = rng.standard_normal((m, nrhs))
        prec = precs[k % len(precs)]
        out.append(serve.Request(k, 0.0, pid, specs[pid][0], N, V, prec))
    return out


def test_device_build_matches_generator(cuda):
    from paper_0912_3678_gb300 import serve
    p = gen.bvp_problem(8, 3, seed_rep=7)
    b = gen.trapezoidal_babd(p, 500)
    spec = serve.BvpSpec(p.Smat, p.K, p.B0, p.B1)
    S, R, B0, B1 = (to_host(t) for t in serve.build_bvp_device(spec, 500, cuda))
    rhs, yex = serve.build_rhs_device(spec, 500, p.V, cuda)
    assert np.abs(S - b.S).max() <= 1e-15 and np.abs(R - b.R).max() <= 1e-15
    assert np.abs(to_host(rhs) - b.RHS).max() <= 1e-13 * np.abs(b.RHS).max()
    assert np.abs(to_host(yex) - b.Yexact).max() <= 1e-14


def test_alone_equals_mix_and_oracle(cuda):
    from paper_0912_3678_gb300 import serve
    reqs = _requests()
    alone = []
    for r in reqs:
        srv = serve.Server(cuda, streams=1, cache=False)
        srv.submit(r)
        srv.drain()
        assert r.status == 0
        alone.append(to_host(r.Y))
        srv.close()
    mix_reqs = _requests()
    srv = serve.Server(cuda, streams=4)
    for r in mix_reqs:
        srv.submit(r)
    srv.drain()
    st = srv.stats()
    assert st["failed"] == 0 and st["cache_hits"] >= 1
    for r, ya in zip(mix_reqs, alone):
        ym = to_host(r.Y)
        assert oracle.rel_err(ym, ya) <= 1e-11, r.rid
        b = gen.trapezoidal_babd(gen.BvpProblem(r.spec.S, r.spec.K, r.spec.B0, r.spec.B1, r.V), r.N)
        ref = oracle.babd_solve(b.S, b.R, b.B0, b.B1, b.RHS)
        tol = 1e-11 if r.prec == "fp64" else 1e-10
        assert oracle.rel_err(ym, ref) <= tol, (r.rid, r.prec)
    srv.close()


def test_memory_admission_respects_cap(cuda):
    from paper_0912_3678_gb300 import serve
    reqs = _requests(8, seed=3, precs=("fp64",))
    probe = serve.Server(cuda, streams=1)
    cap = int(1.5 * max(probe.footprint(r) for r in reqs))   # about one request at a time
    srv = serve.Server(cuda, mem_cap_bytes=cap, streams=4, cache=False)
    for r in reqs:
        srv.submit(r)
    srv.drain()
    assert srv.stats()["failed"] == 0
    assert srv.peak_in_use <= cap
    srv.close()
    # a request larger than the cap is refused at once (BT_ERR_NOMEM), not queued forever
    tiny = serve.Server(cuda, mem_cap_bytes=1 << 20, streams=2)
    r = _requests(1, seed=4, precs=("fp64",))[0]
    tiny.submit(r)
    tiny.drain(timeout_s=30)
    assert r.status == 2
    tiny.close()


def test_cache_hit_under_memory_pressure_keeps_its_factorization(cuda):
    """A repeated problem arrives when the cache must shed memory: the eviction
    releases another idle factorization, never the one the request reuses.
    A (4 RHS) and C (1 RHS) stay cached; the cap leaves no room for B's vectors
    (B repeats A with 4 RHS) unless one of them goes."""
    from paper_0912_3678_gb300 import serve
    rng = np.random.default_rng(5)
    pa = gen.bvp_problem(8, 1, seed_rep=501)
    pc = gen.bvp_problem(8, 1, seed_rep=502)
    sa = serve.BvpSpec(pa.Smat, pa.K, pa.B0, pa.B1)
    sc = serve.BvpSpec(pc.Smat, pc.K, pc.B0, pc.B1)
    A = serve.Request(0, 0.0, 0, sa, 800, rng.standard_normal((8, 4)), "fp64")
    C = serve.Request(1, 0.0, 1, sc, 800, rng.standard_normal((8, 1)), "fp64")
    B = serve.Request(2, 0.0, 0, sa, 800, rng.standard_normal((8, 4)), "fp64")
    probe = serve.Server(cuda, streams=1)
    wsA, mat, vecB = probe._footprint(B, serve._round_nrhs(4))
    wsC, _, _ = probe._footprint(C, serve._round_nrhs(1))
    probe.close()
    cap = (wsA + mat) + (wsC + mat) + vecB - 1
    srv = serve.Server(cuda, mem_cap_bytes=cap, streams=1)
    for r in (A, C):
        srv.submit(r)
        srv.drain(timeout_s=60)
    assert len(srv.cache) == 2
    srv.submit(B)
    srv.drain(timeout_s=60)
    assert B.status == 0 and B.cache_hit
    assert len(srv.cache) == 1
    b = gen.trapezoidal_babd(gen.BvpProblem(sa.S, sa.K, sa.B0, sa.B1, B.V), B.N)
    ref = oracle.babd_solve(b.S, b.R, b.B0, b.B1, b.RHS)
    assert oracle.rel_err(to_host(B.Y), ref) <= 1e-11
    srv.close()


def test_trace_replay_reports_latency(cuda):
    from paper_0912_3678_gb300 import serve
    trace = gen.serve_trace(0.05, rate=400.0, ms=(4, 8), Nmin=200, Nmax=2000, reuse=0.3, rep=1)
    reqs = serve.requests_from_trace(trace)
    srv = serve.Server(cuda, streams=4)
    st = srv.run_trace(reqs, realtime=True, timeout_s=120)
    assert st["requests"] == len(reqs) and st["failed"] == 0
    assert 0 < st["p50_ms"] <= st["p99_ms"]
    srv.close()


def test_refined_request_that_does_not_converge_falls_back_to_fp64(cuda):
    """With no refinement sweep the FP32-factor solution fails the backward-error
    test (BT_ERR_NOT_CONVERGED); the server queues the request again as FP64 and
    returns that solution instead of a failure."""
    from paper_0912_3678_gb300 import serve
    reqs = _requests(count=6, seed=3, precs=("fp32_ir",))
    srv = serve.Server(cuda, streams=2, sweeps=0)
    for r in reqs:
        srv.submit(r)
    srv.drain()
    st = srv.stats()
    assert st["failed"] == 0
    assert st["fp64_fallbacks"] == len(reqs)
    for r in reqs:
        assert r.fallback and r.prec == "fp64" and r.status == 0
        b = gen.trapezoidal_babd(gen.BvpProblem(r.spec.S, r.spec.K, r.spec.B0, r.spec.B1, r.V), r.N)
        ref = oracle.babd_solve(b.S, b.R, b.B0, b.B1, b.RHS)
        assert oracle.rel_err(to_host(r.Y), ref) <= 1e-11, r.rid
    srv.close()
