"""Benchmark of the partition-method solver on one GB300 (or N replicas).

Default workload: block tridiagonal A x = f with m = 16 blocks, N = 16384 block
rows (n = 262144 unknowns) and 8 right-hand sides; D_j = 4I + G/4, B_j, C_j =
G/4 (seeded synthetic data).  One step = the whole hot path on one system:
factor (local block LU with spikes, reduced systems, recursion) + solve, for
three paths: "fp64" (every step in FP64), "fp32_ir" (FP32 local factors, FP64
reduced-system factorization, refinement with a double-float residual) and
"bf16_ir" (as fp32_ir with BF16 tensor-core Schur products).  The headline
value is the faster path whose normwise relative error against the FP64
oracle is <= 1e-10.  Metric: unknowns x right-hand sides solved per second.
The same JSON line carries, under "configs", short runs of the other
workloads (1024 scalar systems of n = 2^16, the BABD boundary value problem,
the 4096 uneven systems and the served stream with p50/p99 latency);
--no-configs leaves them out.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                  [--workload block16|block|babd8|scalar|scalar_batch|batch|serve|pivot|parareal|cyclic]
                  [--tuning key=value,...]

The device figure (`value`) times one captured CUDA graph per step with the
inputs already in device memory and L2 flushed between steps; `e2e` times the
same step from pinned host arrays through the library's host-array entry
point (bt_plan_capture_host + replay: block rows copied in slabs while the
level-0 factorization runs, X copied back) for block tridiagonal workloads,
otherwise host copies around the captured step.  --impl reference times the
FP64 CPU oracle on the same workload (the baseline of this project).  With
N > 1 (torchrun), every rank solves its own replica (replicas only, weak
scaling); timings are max over ranks.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "unknowns solved/s at rel err <=1e-10 vs plain FP64"
UNIT = "unknowns*rhs/s"
FP64_PEAK_TFLOPS = 152 * 2 * 2 * 2.07e9 / 1e12   # 152 SMs x 2 DFMA/clk x 2 flop x 2.07 GHz


def _hbm_peak_gbs():
    """Measured device copy bandwidth of this GPU model (MEASURED_PEAKS.json), else 6800 GB/s."""
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            return float(json.load(fh)["hbm_gbs"])
    except (OSError, KeyError, ValueError):
        return 6800.0


HBM_PEAK_GBS = _hbm_peak_gbs()


def _workload(name: str, m_opt=None, N_opt=None, nr_opt=None):
    import gen
    if name == "block":
        N, m, nr = N_opt or 16384, m_opt or 16, nr_opt or 8
        s = gen.btri_random(N, m, nr, seed_rep=0)
        return dict(kind="btri", N=N, m=m, nrhs=nr, sys=s, unknowns=N * m * nr,
                    desc=f"block tridiagonal m={m}, N={N} block rows (n={N * m}), {nr} RHS; D=4I+G/sqrt(m), B,C=G/sqrt(m)")
    if name == "block16":
        N, m, nr = 16384, 16, 8
        s = gen.btri_random(N, m, nr, seed_rep=0)
        return dict(kind="btri", N=N, m=m, nrhs=nr, sys=s, unknowns=N * m * nr,
                    desc="block tridiagonal m=16, N=16384 block rows (n=262144), 8 RHS; D=4I+G/4, B,C=G/4")
    if name == "babd8":
        N, m, nr = 1 << 18, 8, 1
        b = gen.babd_bvp(N, m, nr, seed_rep=0)
        return dict(kind="babd", N=N, m=m, nrhs=nr, sys=b, unknowns=(N + 1) * m * nr,
                    desc="BABD trapezoidal BVP m=8, N=2^18 steps (n=2097160), 1 RHS")
    if name == "scalar":
        n = 1 << 16
        t = gen.tri_sdd(n, 1, seed_rep=0)
        s = gen.BtriSystem(t.dl.reshape(n, 1, 1), t.d.reshape(n, 1, 1), t.du.reshape(n, 1, 1), t.f, t.xstar)
        return dict(kind="btri", N=n, m=1, nrhs=1, sys=s, unknowns=n,
                    desc="scalar tridiagonal n=2^16, d~U[4,6], dl,du~U[-1,1], 1 RHS")
    raise SystemExit(f"unknown workload {name}")


# DRAM bytes (read + written) per launch of the dominant kernel, from one ncu
# capture of that launch in the same configuration (workload, path, kernel,
# level-0 partitions): profiles/factor_cta_fp64_m16_block16.md.  Any other
# configuration reports null; an entry is dropped when its kernel changes.
# Estimated forward-error target of the refined paths' stopping test (the metric
# asks for 1e-10 against FP64; the result is also checked against the oracle).
FWD_TARGET = 1e-11

MEASURED_TRAFFIC = {
    ("block16", "fp64", "factor", 608): 150.0e6,
    # the split-copy residual's traffic does not depend on the partitioning (any p0)
    ("block16", "fp32_ir", "residual", None): 141.6e6,
}


def _measured_traffic(workload, path, kernel, p0):
    """ncu DRAM bytes of one launch (profiles/), or None when not captured."""
    v = MEASURED_TRAFFIC.get((workload, path, kernel, p0))
    return v if v is not None else MEASURED_TRAFFIC.get((workload, path, kernel, None))


def _cpu_info():
    """Host CPU model and the cores this process may use."""
    model = None
    try:
        with open("/proc/cpuinfo") as fh:
            for ln in fh:
                k = ln.split(":")[0].strip().lower()
                if k in ("model name", "cpu model", "processor name"):
                    model = ln.split(":", 1)[1].strip()
                    break
    except OSError:
        pass
    if model is None:
        try:
            out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=5).stdout
            for ln in out.splitlines():
                if ln.lower().startswith("model name"):
                    model = ln.split(":", 1)[1].strip()
                    break
        except (OSError, subprocess.SubprocessError):
            pass
    if model is None:
        import platform
        model = platform.processor() or platform.machine()
    try:
        ncpu = len(os.sched_getaffinity(0))
    except AttributeError:
        ncpu = os.cpu_count()
    return {"cpu_model": model, "nproc": ncpu}


def _derived_peaks(dev, sm_mhz):
    """FP64 and FP32 FMA peaks (TFLOP/s) from this device's SM count and the SM
    clock sampled during the timed region (2 FP64 and 128 FP32 FMA per clock
    per SM on this GPU; one FMA = 2 flop)."""
    import torch
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    ghz = (sm_mhz or 2070.0) / 1e3
    return {"sms": sms, "sm_ghz": ghz, "fp64": sms * 2 * 2 * ghz / 1e3, "fp32": sms * 128 * 2 * ghz / 1e3}


def _factor_flops_per_row(m: int) -> float:
    # algorithmic count per local block row: block-Thomas factorization
    # (2/3 + 2 + 2) m^3 plus the left spike 4 m^3
    return (2.0 / 3.0 + 2.0 + 2.0 + 4.0) * m ** 3


def _clock_sampler(stop_evt, out_rows):
    cmd = ["nvidia-smi",
           "--query-gpu=index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
           "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
           "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap",
           "--format=csv,noheader,nounits", "-lms", "100"]
    try:
        idx = os.environ.get("CUDA_VISIBLE_DEVICES", "")
        p = subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
    except Exception:
        return
    try:
        while not stop_evt.is_set():
            line = p.stdout.readline()
            if not line:
                break
            out_rows.append(line.strip())
    finally:
        p.terminate()
        try:
            p.wait(timeout=2)
        except Exception:
            p.kill()


def _clocks_summary(rows, local_rank=0):
    vals, mx, reasons = [], None, set()
    names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
    for r in rows:
        f = [x.strip() for x in r.split(",")]
        if len(f) < 9:
            continue
        try:
            if int(f[0]) != local_rank and len(rows) > 0:
                pass
            vals.append(float(f[1]))
            mx = float(f[2])
        except ValueError:
            continue
        for nm, v in zip(names, f[5:9]):
            if v.lower().startswith("active"):
                reasons.add(nm)
    if not vals:
        return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
    return {"sm_mhz": statistics.median(vals), "sm_max_mhz": mx, "reasons": sorted(reasons),
            "samples": len(vals)}


def _dist():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def run_reference(args):
    ws, rank, _ = _dist()
    if rank != 0:
        return 0
    import oracle
    w = _workload(args.workload, args.m, args.N, args.nrhs)
    s = w["sys"]

    def step():
        if w["kind"] == "btri":
            return oracle.btri_solve(s.B, s.D, s.C, s.F)
        return oracle.babd_solve(s.S, s.R, s.B0, s.B1, s.RHS)

    for _ in range(args.warmup):
        step()
    t = []
    for _ in range(args.steps):
        t0 = time.perf_counter()
        step()
        t.append(time.perf_counter() - t0)
    ms = 1e3 * sum(t) / len(t)
    val = w["unknowns"] / (ms / 1e3)
    line = {
        "impl": "reference", "metric": METRIC, "value": val, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": w["desc"], "path": "sequential FP64 oracle (block Thomas / BABD GEPP), 1 core"},
        "cpu_baseline": {"value": val, "unit": UNIT, "cores": 1, "kind": "oracle",
                         "sample": f"the full workload, {args.steps} timed solves", **_cpu_info()},
        "e2e": {"value": val, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line))
    return 0


def run_batch(args, emit=True):
    """Batched workload: 4096 uneven independent systems (n log-uniform, m from {1,4,8,16,32},
    50/50 FP64 / BF16+refinement), generated on the device, one graph launch
    per step.  Accuracy: a sample of systems against the oracle."""
    import torch

    import gen
    import paper_0912_3678_gb300 as bt
    from paper_0912_3678_gb300 import build as _build
    _build.build()
    dev = torch.device("cuda:0")
    scalar = args.workload == "scalar_batch"
    specs = gen.scalar_batch_specs() if scalar else gen.batch_specs(args.batch_count, nmax=args.batch_nmax)
    systems = gen.batch_systems_device(specs, dev)
    unknowns = sum(sd["F"].shape[0] for sd in systems)
    torch.cuda.synchronize()
    from paper_0912_3678_gb300 import tune
    cap = int(args.batch_memcap_gb * 2 ** 30)
    if args.no_tune:
        k0, ktimes = 32, {}
    else:
        k0, ktimes = tune.tune_batch(systems, ir_sweeps=4, mem_cap_bytes=cap)
    t0 = time.perf_counter()
    b = bt.BtBatch(systems, ir_sweeps=4, mem_cap_bytes=cap, tuner=tune.batch_tuner(k0))
    t_create = time.perf_counter() - t0
    waves, nodes, nbytes = b.info()
    for _ in range(args.warmup):
        b.run()
    b.finish()
    ev = []
    torch.cuda.synchronize()
    for _ in range(args.steps):
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record()
        b.run()
        e1.record()
        ev.append((e0, e1))
    torch.cuda.synchronize()
    ms = sum(a.elapsed_time(c) for a, c in ev) / len(ev)
    code, status, rel = b.finish()
    # accuracy on a sample against the oracle
    import numpy as np
    import oracle
    rng = np.random.default_rng(0)
    sample = sorted(rng.choice(len(systems), size=min(24, len(systems)), replace=False).tolist())
    worst = {"fp64": 0.0, "bf16_ir": 0.0}
    t_or, n_or = 0.0, 0
    for k in sample:
        sd = systems[k]
        if sd["D"].numel() > 3e7:
            continue
        h = {n: sd[n].cpu().numpy() for n in ("B", "D", "C", "F", "X")}
        t1 = time.perf_counter()
        ref = oracle.btri_solve(h["B"], h["D"], h["C"], h["F"])
        t_or += time.perf_counter() - t1
        n_or += h["F"].size
        worst[sd["prec"]] = max(worst[sd["prec"]], oracle.rel_err(h["X"], ref))
    if scalar:
        desc = (f"{len(systems)} independent scalar tridiagonal systems, n=2^16 each, d~U[4,6], "
                f"dl,du~U[-1,1], 1 RHS, FP64, one batch")
        # Both rooflines of the one-shot scalar solve: 40 algorithmic bytes per unknown (read
        # dl, d, du, f; write x) and 15 algorithmic FP64 flops per unknown (the partition
        # method's LU 3, spikes 3, forward and back substitution 5, spike corrections 4).
        # At about 0.4 flop per byte, far above the FP64/HBM balance of this GPU (about
        # 0.18 flop per byte), the FP64 pipe binds.
        per_s = unknowns / (ms / 1e3)
        gbs = 40.0 * per_s / 1e9
        ach = 15.0 * per_s / 1e12
        pk = _derived_peaks(dev, None)
        roof = {"bound": "alu", "achieved": ach, "peak": pk["fp64"], "unit": "TFLOP/s",
                "frac": ach / pk["fp64"], "traffic": None,
                "kernel": "whole step (factor + solve, all levels), 15 FP64 flop per unknown",
                "peak_source": f"derived: {pk['sms']} SMs x 2 FP64 FMA/clk x 2 flop x 2.07 GHz (maximum clock)",
                "hbm": {"achieved": gbs, "peak": HBM_PEAK_GBS, "unit": "GB/s", "frac": gbs / HBM_PEAK_GBS,
                        "bytes_per_unknown": 40}}
    else:
        desc = (f"{len(systems)} uneven block tridiagonal systems, n log-uniform "
                f"[1e3,{args.batch_nmax:g}], m in {{1,4,8,16,32}}, 50/50 FP64 / BF16+IR, 1 RHS")
        roof = None
    line = {"metric": METRIC, "value": unknowns / (ms / 1e3), "unit": "unknowns/s", "n_gpus": 1,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None,
            "dtype": "f64" if scalar else "f64 + bf16/f32+f64 refinement", "data": "synthetic",
            "config": {"workload": desc,
                       "graph_nodes": nodes, "waves": waves, "workspace_gb": nbytes / 2 ** 30,
                       "create_s": t_create, "partition_rows": k0,
                       "tuning_ms": {str(k): v for k, v in ktimes.items()}},
            "statuses_ok": sum(1 for x in status if x == 0), "systems": len(status),
            "rel_err_sample_max": worst, "roofline": roof,
            "cpu_baseline": {"value": n_or / t_or if t_or else None, "unit": "unknowns/s", "cores": 1,
                             "kind": "oracle", "sample": f"{len(sample)} systems of the batch", **_cpu_info()}}
    if emit:
        print(json.dumps(line))
    b.close()
    del b, systems
    torch.cuda.empty_cache()
    return line


def _timed(step, warmup, steps):
    """Mean ms per step on the current stream (CUDA events), after warm-up."""
    import torch
    for _ in range(warmup):
        step()
    torch.cuda.synchronize()
    ev = []
    for _ in range(steps):
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record()
        step()
        e1.record()
        ev.append((e0, e1))
    torch.cuda.synchronize()
    return sum(a.elapsed_time(b) for a, b in ev) / len(ev)


def run_pivot(args):
    """Pivoted partitions (bt_tuning.pivot): a non-dominant scalar tridiagonal
    system with 2 % exactly zero diagonal entries, n = 2^20, one factor +
    solve per step (the factorization splits partitions at the breakdowns).
    Accuracy: normwise backward error, and the oracle's dense GEPP is out of
    reach, so the CPU baseline is the oracle's Thomas algorithm on the
    dominant system of the same size."""
    import numpy as np
    import torch

    import gen
    import paper_0912_3678_gb300 as bt
    from paper_0912_3678_gb300 import build as _build
    _build.build()
    dev = torch.device("cuda:0")
    N, m = 1 << 20, 1
    s = gen.btri_nondominant(N, m, 1, seed_rep=0, zero_frac=0.02)
    B, D, C, F = (torch.from_numpy(np.ascontiguousarray(a)).to(dev) for a in (s.B, s.D, s.C, s.F))
    X = torch.empty_like(F)
    # level-0 partition count: more partitions shorten the local factorizations and
    # lengthen the enlarged reduced system (solved by one warp); time a few and keep the best
    trials = {}
    for p0 in (1024, 2048, 4096, 8192):
        with bt.BtPlan.tuned(N, m, 1, "fp64", {"p0": p0, "pivot": 1}) as cand:
            def cstep():
                cand.factor(B, D, C)
                cand.solve(F, X)
            trials[p0] = _timed(cstep, 2, 3)
    p0 = min(trials, key=trials.get)
    plan = bt.BtPlan.tuned(N, m, 1, "fp64", {"p0": p0, "pivot": 1})

    def step():
        plan.factor(B, D, C)
        plan.solve(F, X)
    ms = _timed(step, args.warmup, args.steps)
    p_eff = plan.levels()[0][1]
    Xh = X.cpu().numpy()
    R = s.F - gen.btri_matvec(s.B, s.D, s.C, Xh)
    rows = np.abs(s.D).sum(2)
    rows[1:] += np.abs(s.B[1:]).sum(2)
    rows[:-1] += np.abs(s.C[:-1]).sum(2)
    eta = np.abs(R).max() / (rows.max() * np.abs(Xh).max() + np.abs(s.F).max())
    plan.close()
    line = {"metric": METRIC, "value": N * m / (ms / 1e3), "unit": "unknowns/s", "n_gpus": 1, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": "pivoted partitions: non-dominant scalar tridiagonal n=2^20, 2% zero diagonal "
                                   "entries", "p0": p0, "p0_trials_ms": {str(k): v for k, v in trials.items()},
                       "partitions_after_splits": p_eff,
                       "launch": "kernel by kernel (the factorization synchronises per splitting pass)"},
            "backward_error": float(eta)}
    print(json.dumps(line))
    return 0


def run_parareal(args):
    """Parareal (ivp_parareal) for the 1-D heat equation y' = L y + g0 + t g1,
    n = 2^18 interior points, smooth data (four Fourier modes), T = 0.05,
    p = 32 coarse intervals of 16 trapezoidal steps, one backward Euler coarse
    step; iterated until the iterates change by at most 1e-10 (relative; for this stiff
    problem, h/2 |lambda_max| ~ 7e6, the change of the iterates stalls near 2e-12, the
    rounding level of the propagators, so a tolerance of 1e-12 would never be met
    reliably).  Throughput =
    space-time unknowns of the fine grid (n p nfine) per second.  Accuracy and
    the CPU baseline: the oracle's sequential fine integration."""
    import numpy as np
    import torch

    import paper_0912_3678_gb300 as bt
    from paper_0912_3678_gb300 import build as _build
    _build.build()
    dev = torch.device("cuda:0")
    n, p, nfine, T = 1 << 18, 32, 16, 0.05
    import gen
    dl, d, du, y0, g0, g1 = gen.heat_problem(n, nu=0.5, seed_rep=0, smooth=True)
    dv = [torch.from_numpy(a).to(dev) for a in (dl, d, du, g0, y0, g1)]
    U = torch.empty((p + 1, n), dtype=torch.float64, device=dev)
    its = [0]

    def step():
        _, it, code, _ = bt.ivp_parareal(dv[0], dv[1], dv[2], dv[3], dv[4], T, p, nfine, 1, kmax=p, tol=1e-10,
                                         g1=dv[5], U=U)
        its[0] = it
    ms = _timed(step, max(1, args.warmup // 3), max(1, args.steps // 4))
    from oracle import ivp          # the CPU baseline and the accuracy check
    t0 = time.perf_counter()
    ref = ivp.sequential_fine(dl, d, du, y0, g0, g1, T, p, nfine)
    t_or = time.perf_counter() - t0
    err = float(np.abs(U.cpu().numpy() - ref).max() / np.abs(ref).max())
    line = {"metric": METRIC, "value": n * p * nfine / (ms / 1e3), "unit": "space-time unknowns/s", "n_gpus": 1,
            "steps": max(1, args.steps // 4), "warmup": max(1, args.warmup // 3), "ms_per_step": ms,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": f"Parareal, heat equation n=2^18 (smooth data, T={T}), p={p}, nfine={nfine}, "
                                   "backward Euler coarse",
                       "iterations": its[0]},
            "rel_err_vs_oracle": err,
            "cpu_baseline": {"value": n * p * nfine / t_or, "unit": "space-time unknowns/s", "cores": 1,
                             "kind": "oracle", "sample": "the sequential fine integration of the same problem"}}
    print(json.dumps(line))
    return 0


def run_cyclic(args):
    """Circulant-like (cyc_*): periodic BVP, trapezoidal rule, m = 8, N = 2^18
    steps, one factor + solve per step; accuracy and CPU baseline: the
    oracle's BABD elimination of the same discretisation with y_N kept."""
    import numpy as np
    import torch

    import gen
    import oracle
    import paper_0912_3678_gb300 as bt
    from paper_0912_3678_gb300 import build as _build
    _build.build()
    dev = torch.device("cuda:0")
    N, m = 1 << 18, 8
    s = gen.periodic_bvp(N, m, 1, seed_rep=0)
    S, R, RHS = (torch.from_numpy(np.ascontiguousarray(a)).to(dev) for a in (s.S, s.R, s.RHS))
    Y = torch.empty_like(RHS)
    plan = bt.CycPlan(N, m, 1)

    def step():
        plan.factor(S, R)
        plan.solve(RHS, Y)
    ms = _timed(step, args.warmup, args.steps)
    plan.close()
    t0 = time.perf_counter()
    ref = oracle.babd_solve(s.S, s.R, np.eye(m), -np.eye(m), np.concatenate([np.zeros((m, 1)), s.RHS]))[:N * m]
    t_or = time.perf_counter() - t0
    line = {"metric": METRIC, "value": N * m / (ms / 1e3), "unit": "unknowns/s", "n_gpus": 1, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": "circulant-like: periodic trapezoidal BVP m=8, N=2^18 (cyclic block bidiagonal)",
                       "launch": "kernel by kernel"},
            "rel_err_vs_oracle": float(oracle.rel_err(Y.cpu().numpy(), ref)),
            "cpu_baseline": {"value": N * m / t_or, "unit": "unknowns/s", "cores": 1, "kind": "oracle",
                             "sample": "the full workload once"}}
    print(json.dumps(line))
    return 0


def run_serve(args, emit=True):
    """Served workload: Poisson arrivals of BVP solves (m in {4,8,16}, N log-uniform
    [1e3, 5e5], 1-32 RHS, 30% factorization reuse) replayed in real time."""
    import torch

    import gen
    from paper_0912_3678_gb300 import build as _build
    from paper_0912_3678_gb300 import serve
    _build.build()
    dev = torch.device("cuda:0")
    warm = serve.requests_from_trace(gen.serve_trace(0.05, rate=200, rep=7), prec=args.serve_prec)
    srv = serve.Server(dev, mem_cap_bytes=150e9, streams=8)
    srv.run_trace(warm, realtime=False)
    srv.close()
    trace = gen.serve_trace(args.serve_seconds, rate=args.serve_rate, rep=0)
    reqs = serve.requests_from_trace(trace, prec=args.serve_prec)
    srv = serve.Server(dev, mem_cap_bytes=150e9, streams=8)
    st = srv.run_trace(reqs, realtime=True, timeout_s=1800)
    srv.close()
    line = {"metric": METRIC, "value": st["unknowns_per_s"], "unit": "unknowns*rhs/s", "n_gpus": 1,
            "steps": st["requests"], "warmup": len(warm), "ms_per_step": st["mean_ms"], "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": args.serve_prec, "data": "synthetic",
            "config": {"workload": f"served BVP stream, Poisson {args.serve_rate:g} req/s for "
                                   f"{args.serve_seconds:g} s, m in {{4,8,16}}, N log-uniform [1e3,5e5], "
                                   "1-32 RHS, 30% reuse, 150 GB cap, 8 streams"},
            "p50_ms": st["p50_ms"], "p99_ms": st["p99_ms"], "served": st}
    if emit:
        print(json.dumps(line))
    torch.cuda.empty_cache()
    return line


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="block16",
                    choices=["block16", "block", "babd8", "scalar", "scalar_batch", "batch", "serve", "pivot", "parareal",
                             "cyclic"])
    ap.add_argument("--m", type=int, default=None, help="block order of --workload block")
    ap.add_argument("--N", type=int, default=None, help="block rows of --workload block")
    ap.add_argument("--nrhs", type=int, default=None, help="right-hand sides of --workload block")
    ap.add_argument("--batch-count", type=int, default=4096)
    ap.add_argument("--batch-nmax", type=float, default=1e6)
    ap.add_argument("--batch-memcap-gb", type=float, default=80.0)
    ap.add_argument("--serve-seconds", type=float, default=5.0)
    ap.add_argument("--serve-rate", type=float, default=2000.0)
    ap.add_argument("--serve-prec", default="fp64")
    ap.add_argument("--paths", default="fp64,fp32_ir,bf16_ir")
    ap.add_argument("--no-configs", action="store_true",
                    help="headline only: skip the other workloads' summary in the JSON line")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-tune", action="store_true", help="use the built-in partitioning instead of the autotuner")
    ap.add_argument("--tuning", default=None,
                    help="fixed partitioning for every path instead of the autotuner: key=value pairs "
                         "of bt_tuning, e.g. p0=608,reduced=1")
    ap.add_argument("--no-graph", action="store_true", help="launch kernel by kernel instead of one CUDA graph per step")
    args = ap.parse_args()
    args.warmup = max(args.warmup, 3)
    if args.workload == "serve":
        os.environ.setdefault("PYTORCH_CUDA_ALLOC_CONF", "expandable_segments:True")
    if args.impl == "reference":
        return run_reference(args)
    if args.workload in ("batch", "scalar_batch"):
        run_batch(args)
        return 0
    if args.workload == "serve":
        run_serve(args)
        return 0
    if args.workload == "pivot":
        return run_pivot(args)
    if args.workload == "parareal":
        return run_parareal(args)
    if args.workload == "cyclic":
        return run_cyclic(args)

    import torch
    ws, rank, local = _dist()
    dist = None
    if ws > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    dev = torch.device(f"cuda:{local}")
    torch.cuda.set_device(dev)

    from paper_0912_3678_gb300 import build as _build
    if rank == 0 or ws == 1:
        _build.build()
    if dist is not None:
        dist.barrier()
    line = _measure(args, dist, ws, rank, local)
    if rank == 0:
        if args.workload == "block16" and not args.no_configs:
            line["configs"] = _other_configs(args)
        print(json.dumps(line))
    if dist is not None:
        dist.destroy_process_group()
    return 0


def _other_configs(args):
    """The other workloads, each measured briefly after the headline on the
    same GPU (fewer steps, built-in partitioning for the batches): the scalar
    throughput batch, the BABD boundary value problem, the uneven batch and
    the served stream.  One summary per workload: its metric, error against
    the oracle, roofline, and p50/p99 where it has latencies."""
    import copy

    import torch
    keys = ("metric", "value", "unit", "ms_per_step", "steps", "warmup", "dtype", "rel_err_vs_oracle",
            "rel_err_sample_max", "backward_error", "roofline", "cpu_baseline", "p50_ms", "p99_ms", "statuses_ok",
            "systems", "e2e")
    out = {}

    def summary(line, extra=None):
        d = {k: line[k] for k in keys if k in line and line[k] is not None}
        d["workload"] = line.get("config", {}).get("workload")
        if "paths" in line:
            d["paths"] = {p: {k: v for k, v in q.items() if k in ("ms_per_step", "value", "rel_err_vs_oracle")}
                          for p, q in line["paths"].items()}
            d["path"] = line.get("config", {}).get("path")
        if extra:
            d.update(extra)
        return d

    def run(name, fn):
        t0 = time.perf_counter()
        try:
            out[name] = fn()
        except Exception as exc:            # a failed extra leaves the headline intact
            out[name] = {"error": f"{type(exc).__name__}: {exc}"[:300]}
        out[name]["wall_s"] = round(time.perf_counter() - t0, 1)
        torch.cuda.empty_cache()

    def babd():
        a = copy.copy(args)
        a.workload, a.paths, a.tuning, a.cpu_seconds = "babd8", "fp64,fp32_ir", None, 3.0
        return summary(_measure(a, None, 1, 0, int(os.environ.get("LOCAL_RANK", "0"))))

    def batch(scalar):
        a = copy.copy(args)
        a.workload = "scalar_batch" if scalar else "batch"
        a.steps, a.warmup, a.no_tune = 3, 2, True
        return summary(run_batch(a, emit=False), {"tuning": "built-in"})

    def serve(rate, seconds):
        a = copy.copy(args)
        a.serve_rate, a.serve_seconds, a.serve_prec = rate, seconds, "fp64"
        return summary(run_serve(a, emit=False))

    run("scalar_batch_1024x65536", lambda: batch(True))
    run("babd_m8_N262144", babd)
    run("batch_4096_uneven", lambda: batch(False))
    run("serve_2000rps", lambda: serve(2000.0, 1.0))
    run("serve_200rps", lambda: serve(200.0, 2.0))
    return out


def _measure(args, dist, ws, rank, local):
    """One workload, every path of --paths: the timed captured step, the
    end-to-end host-array step, per-kernel times, the roofline of the
    dominant level-0 kernel and (rank 0) the oracle baseline and errors.
    Returns the JSON line (None on ranks other than 0)."""
    import torch
    dev = torch.device(f"cuda:{local}")
    import paper_0912_3678_gb300 as bt
    from paper_0912_3678_gb300 import dist as bdist

    w = _workload(args.workload, args.m, args.N, args.nrhs)
    s = w["sys"]
    N, m, nr = w["N"], w["m"], w["nrhs"]
    stream = torch.cuda.current_stream(dev)

    def dev_t(a):
        return torch.from_numpy(np.ascontiguousarray(a)).to(dev)

    if w["kind"] == "btri":
        mats_h = [s.B, s.D, s.C]
        rhs_h = s.F
        Plan = bt.BtPlan
    else:
        mats_h = [s.S, s.R, s.B0, s.B1]
        rhs_h = s.RHS
        Plan = bt.AbdPlan
    mats = [dev_t(a) for a in mats_h]
    F = dev_t(rhs_h)
    X = torch.empty_like(F)
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device=dev)   # 256 MB > L2

    results = {}
    paths = [p for p in args.paths.split(",") if p]
    tunings = {}
    if w["kind"] == "babd" and args.tuning:
        # BABD plans: {"reduced": 1} = cyclic reduction of the whole system (FP64 only)
        fixed = {k: int(v) for k, v in (kv.split("=") for kv in args.tuning.split(",") if kv)}
        paths = [p for p in paths if p == "fp64"] if fixed.get("reduced") else paths
        for prec in paths:
            tunings[prec] = dict(fixed)
    elif w["kind"] == "btri" and args.tuning:
        fixed = {k: int(v) for k, v in (kv.split("=") for kv in args.tuning.split(",") if kv)}
        for prec in paths:
            tunings[prec] = dict(fixed)
    elif w["kind"] == "btri" and not args.no_tune:
        from paper_0912_3678_gb300 import tune
        tuner = tune.Tuner(os.path.join(ROOT, "paper_0912_3678_gb300", "_build", "tune_cache.json"))
        for prec in paths:
            tunings[prec] = tuner.tune(m, N, prec, nrhs=nr)
    for prec in paths:
        if prec in tunings:
            plan = Plan.tuned(N, m, nrhs_max=nr, prec=prec, tuning=tunings[prec])
        else:
            plan = Plan(N, m, nrhs_max=nr, prec=prec)

        sweeps = [0]
        if prec != "fp64":
            # the metric's accuracy (1e-10 against FP64) as the refinement's target: stop
            # on the correction-ratio forward-error estimate 10 times below it, or on the
            # FP64-level backward error, whichever comes first
            plan.set_forward_tol(FWD_TARGET)

        def step_plain():
            plan.factor(*mats)
            if prec == "fp64":
                plan.solve(F, X)
            else:
                _, it, rc, code = plan.refine(F, X, tol=1e-12, maxit=30, raise_on_error=True)
                sweeps[0] = max(sweeps[0], it)

        for _ in range(args.warmup):
            step_plain()
        torch.cuda.synchronize(dev)
        use_graph = not args.no_graph
        if use_graph:
            if prec == "fp64":
                plan.capture("factor_solve", F, X)
            else:
                plan.capture("factor_refine", F, X, sweeps=sweeps[0])
            step = plan.replay
            for _ in range(2):
                step()
            torch.cuda.synchronize(dev)
        else:
            step = step_plain
        l0 = plan.launches()
        samples = []
        stop_evt = threading.Event()
        rows = []
        th = None
        if rank == 0 or ws == 1:
            th = threading.Thread(target=_clock_sampler, args=(stop_evt, rows), daemon=True)
            th.start()
            time.sleep(0.3)
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize(dev)
        wall0 = time.perf_counter()
        for _ in range(args.steps):
            flush.fill_(1.0)
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            step()
            e1.record(stream)
            samples.append((e0, e1))
        torch.cuda.synchronize(dev)
        if dist is not None:
            dist.barrier()
        wall = time.perf_counter() - wall0
        stop_evt.set()
        if th is not None:
            th.join(timeout=3)
        launches = plan.launches() - l0
        ms_steps = [a.elapsed_time(b) for a, b in samples]
        ms = sum(ms_steps) / len(ms_steps)
        converged = True
        if use_graph and prec != "fp64":
            code, rel = bt.bt_refine_result(plan.handle, 1e-12)
            converged = code == 0
        Xh = X.cpu().numpy().copy()            # the timed path's own result
        # per-kernel times from a traced kernel-by-kernel pass of the same step
        plan.trace(True)
        ntr = 3
        for _ in range(ntr):
            flush.fill_(1.0)
            step_plain()
        torch.cuda.synchronize(dev)
        kinds = {}
        for k in bt.KERNEL_KINDS:
            tot, n = plan.trace_query(k)
            if n:
                kinds[k] = (tot * args.steps / ntr, n)
        f0_ms, f0_n = plan.trace_query("factor", 0)
        r_ms, r_n = plan.trace_query("residual", 0)
        lvl0 = {k: plan.trace_query(k, 0) for k in ("factor", "solve_fwd", "solve_bwd", "residual")}
        plan.trace(False)
        ms_max = bdist.max_over_ranks(ms, dev)
        results[prec] = dict(ms=ms_max, ms_steps=ms_steps, kinds=kinds, f0=(f0_ms, f0_n), resid=(r_ms, r_n),
                             launches=launches / args.steps, X=Xh, clocks=_clocks_summary(rows, local),
                             wall=wall, levels=plan.levels(), graph=use_graph, sweeps=sweeps[0],
                             converged=converged, lvl0=lvl0, ntr=ntr)
        # end to end through the public API with pinned host buffers
        mats_pin = [torch.from_numpy(np.ascontiguousarray(a)).pin_memory() for a in mats_h]
        F_pin = torch.from_numpy(np.ascontiguousarray(rhs_h)).pin_memory()
        X_pin = torch.empty_like(F_pin).pin_memory()
        # block tridiagonal plans: the library's host-buffer entry point (the block rows
        # copied in chunks of partitions whose factorizations start as their rows arrive);
        # otherwise host copies into the bound device arrays around the captured step
        host_api = w["kind"] == "btri"
        if host_api:
            try:
                plan.factor_solve_host(*mats_pin, F_pin, X_pin, sweeps=-1 if prec == "fp64" else sweeps[0])
                torch.cuda.synchronize(dev)
                if use_graph:
                    plan.capture_host(*mats_pin, F_pin, X_pin, sweeps=-1 if prec == "fp64" else sweeps[0])
            except bt.BtError:
                host_api = False

        def e2e_step():
            if host_api:
                if use_graph:
                    plan.replay()
                else:
                    plan.factor_solve_host(*mats_pin, F_pin, X_pin, sweeps=-1 if prec == "fp64" else sweeps[0])
                return
            for d, h in zip(mats, mats_pin):
                d.copy_(h, non_blocking=True)
            F.copy_(F_pin, non_blocking=True)
            step()
            X_pin.copy_(X, non_blocking=True)
        e2e = []
        for it in range(args.warmup + max(3, args.steps // 2)):
            flush.fill_(1.0)
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            e2e_step()
            e1.record(stream)
            torch.cuda.synchronize(dev)
            if it >= args.warmup:
                e2e.append(e0.elapsed_time(e1))
        if host_api:
            # the host path's own solution against the oracle's
            results[prec]["e2e_X"] = X_pin.numpy().copy()
        results[prec]["e2e_path"] = (("bt_plan_capture_host + bt_plan_replay" if use_graph else "bt_factor_solve_host")
                                     + " (host arrays in and out; the block-row copies overlap the level-0 "
                                     "factorization)" if host_api else "host copies + captured step")
        e2e_ms = sum(e2e) / len(e2e)
        results[prec]["e2e_ms"] = bdist.max_over_ranks(e2e_ms, dev)
        results[prec]["h2d"] = sum(int(a.nbytes) for a in mats_h) + int(rhs_h.nbytes)
        results[prec]["d2h"] = int(rhs_h.nbytes)
        plan.close()

    if rank != 0:
        return None

    # ---- CPU baseline: the oracle on the host cores, bounded sample; its
    # solution also gives each path's error against plain FP64.
    cpu = None
    ref = None
    if not args.no_cpu_baseline:
        import oracle
        def oracle_solve():
            if w["kind"] == "btri":
                return oracle.btri_solve(s.B, s.D, s.C, s.F)
            return oracle.babd_solve(s.S, s.R, s.B0, s.B1, s.RHS)
        t0 = time.perf_counter()
        ref = oracle_solve()
        first = time.perf_counter() - t0
        reps = max(1, min(50, int(getattr(args, "cpu_seconds", 10.0) / max(first, 1e-3))))
        t0 = time.perf_counter()
        for _ in range(reps):
            oracle_solve()
        per = (time.perf_counter() - t0) / reps
        cpu = {"value": w["unknowns"] / per, "unit": UNIT, "cores": 1, "kind": "oracle",
               "sample": f"the full workload solved {reps + 1} times (about {per * (reps + 1):.1f} s), "
                         "single-threaded C, FP64", **_cpu_info()}

    import oracle as _o
    for prec, r in results.items():
        r["rel_err"] = _o.rel_err(r["X"], ref) if ref is not None else None
        if "e2e_X" in r:
            r["e2e_rel_err"] = _o.rel_err(r["e2e_X"], ref) if ref is not None else None
    ok = {p: r for p, r in results.items() if (r["rel_err"] is None or r["rel_err"] <= 1e-10) and r["converged"]}
    head = min(ok, key=lambda p: ok[p]["ms"]) if ok else min(results, key=lambda p: results[p]["ms"])
    r = results[head]
    value = ws * w["unknowns"] / (r["ms"] / 1e3)
    # roofline of the dominant level-0 kernel of the headline path (largest
    # time per step among factor / forward solve / back substitution / FP64
    # residual), on its algorithmic flop count and the peak of its arithmetic
    pk = _derived_peaks(dev, (r["clocks"] or {}).get("sm_mhz"))
    fp64_peak, fp32_peak = pk["fp64"], pk["fp32"]
    if w["kind"] == "btri":
        local_rows = N - (r["levels"][0][1] - 1)
    else:
        local_rows = N - r["levels"][0][1]
    refined = head != "fp64"
    if w["kind"] == "btri":
        flops_per = {
            "factor": _factor_flops_per_row(m) * local_rows,          # (2/3+2+2) m^3 + 4 m^3 per local row
            "solve_fwd": 6.0 * m * m * nr * local_rows,                # 2 matvecs + top-row sweep per row
            "solve_bwd": 4.0 * m * m * nr * local_rows,                # 2 matvecs per row
            # FP64 residual: 3 m^2 nrhs FMA per block row.  Refined paths: the same terms in
            # double-float arithmetic on the FP32 pipe, 15 FP32 flop per term (TwoProduct
            # 1 FMUL + 1 FMA, two cross-term FMAs, TwoSum 6 FADD, 2 FADD into the second sum)
            "residual": (15.0 if refined else 2.0) * 3 * m * m * nr * N,
        }
        bytes_per = {"residual": 8.0 * (3 * m * m * N + 3 * N * m * nr)}   # A, x, f read; r written
    elif (tunings.get(head) or {}).get("reduced"):
        pairs = N // 2                                                  # first cyclic-reduction level
        flops_per = {
            "factor": (2.0 / 3.0 + 2.0 + 2.0) * m ** 3 * pairs,        # LU of R_2k, R^-1 S_2k, S_2k+1 T
            "solve_fwd": 4.0 * m * m * nr * pairs,                     # R^-1 r_2k, S_2k+1 u
            "solve_bwd": 2.0 * m * m * nr * pairs,                     # T y_2k
            "residual": (15.0 if refined else 2.0) * 2 * m * m * nr * (N + 1),
        }
        bytes_per = {"residual": 8.0 * (2 * m * m * N + 3 * (N + 1) * m * nr)}
    else:
        flops_per = {
            "factor": (2.0 / 3.0 + 4.0) * m ** 3 * local_rows,         # LU of R_j, propagator, spike product
            "solve_fwd": 4.0 * m * m * nr * local_rows,                # 2 matvecs per step
            "solve_bwd": 2.0 * m * m * nr * local_rows,                # 1 matvec per step
            "residual": (15.0 if refined else 2.0) * 2 * m * m * nr * (N + 1),
        }
        bytes_per = {"residual": 8.0 * (2 * m * m * N + 3 * (N + 1) * m * nr)}
    cand = {k: v for k, v in r["lvl0"].items() if v[1] > 0}
    roof = None
    if cand:
        dom = max(cand, key=lambda k: cand[k][0])
        t_launch = cand[dom][0] / cand[dom][1] / 1e3
        is64 = not refined
        peak = fp64_peak if is64 else fp32_peak
        ach = flops_per[dom] / t_launch / 1e12
        what = ("FP64" if is64 else ("FP32 double-float" if dom == "residual" else "FP32"))
        roof = {"bound": "alu", "achieved": ach, "peak": peak, "unit": "TFLOP/s", "frac": ach / peak,
                "traffic": _measured_traffic(args.workload, head, dom, r["levels"][0][1]),
                "kernel": f"level-0 {dom} ({what})",
                "peak_source": (f"derived: {pk['sms']} SMs x {2 if is64 else 128} {'FP64' if is64 else 'FP32'} "
                                f"FMA/clk x 2 flop x {pk['sm_ghz']:.3f} GHz (median SM clock sampled during "
                                f"the timed steps)"),
                "launch_ms": t_launch * 1e3}
        if dom in bytes_per:
            gbs = bytes_per[dom] / t_launch / 1e9
            roof["hbm"] = {"achieved": gbs, "peak": HBM_PEAK_GBS, "unit": "GB/s", "frac": gbs / HBM_PEAK_GBS,
                           "bytes_per_launch": bytes_per[dom], "peak_source": "MEASURED_PEAKS.json hbm_gbs"}
    st = sorted(r["ms_steps"])
    p50 = float(np.percentile(st, 50)) if st else None
    p99 = float(np.percentile(st, 99)) if st else None
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": r["ms"], "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64" if head == "fp64" else "f32+f64",
        "data": "synthetic", "p50_ms": p50, "p99_ms": p99,
        "config": {"workload": w["desc"], "path": head, "l2": "flushed (256 MB write) between timed steps",
                   "parallelism": f"replicas x{ws}", "levels": r["levels"],
                   "tuning": tunings.get(head, "built-in"),
                   "launch": "one CUDA graph per step" if r["graph"] else "kernel by kernel",
                   "refinement_sweeps": r["sweeps"] if head != "fp64" else 0,
                   "refinement_stop": (None if head == "fp64" else
                                       f"estimated forward error <= {FWD_TARGET:g} (correction ratio) or "
                                       "backward error <= 4(3m+1)u, checked on the captured step")},
        "roofline": roof,
        "cpu_baseline": cpu,
        "e2e": {"value": ws * w["unknowns"] / (r["e2e_ms"] / 1e3), "unit": UNIT, "h2d_bytes_per_step": r["h2d"],
                "d2h_bytes_per_step": r["d2h"], "path": r.get("e2e_path"),
                "rel_err_vs_oracle": r.get("e2e_rel_err")},
        "clocks": r["clocks"],
        "gpu_launches": r["launches"],
        "rel_err_vs_oracle": r["rel_err"],
        "paths": {p: {"ms_per_step": q["ms"], "value": ws * w["unknowns"] / (q["ms"] / 1e3),
                      "rel_err_vs_oracle": q["rel_err"], "e2e_ms": q["e2e_ms"],
                      "kernel_ms_per_step": {k: v[0] / args.steps for k, v in q["kinds"].items()},
                      "graph": q["graph"], "converged": q["converged"],
                      "launches_per_step": q["launches"]} for p, q in results.items()},
    }
    return line


if __name__ == "__main__":
    sys.exit(main())
