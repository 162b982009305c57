"""Continuous-batching server for linear BVP solves (BABD systems, Sec. 3) on
one GPU.

Requests arrive over time (``submit``); the scheduler (``poll``) admits them
while their HBM footprint fits under the cap and a stream slot is free, runs
each admitted request on its own CUDA stream (problem build, ``abd_factor``
unless the factorization is cached, ``abd_solve`` or asynchronous FP64
refinement), and retires requests whose completion event has fired, freeing
their memory so queued ones can start.  Work of different requests overlaps
on the device.  Factorizations are cached by problem id (LRU, evicted when
memory is needed); a hit only solves.  Plans are built on workspace from
torch's caching allocator, so steady-state serving makes no cudaMalloc call.

The problem of a request is the trapezoidal discretisation of
y' = L(t) y + q(t), L(t) = S + cos(2 pi t) K, with boundary rows B0, B1 and
the manufactured solution y(t) = exp(sin 3t) v (one v per right-hand side),
built on the device from the compact description (S, K, B0, B1, v) -- the
same recipe as ``gen.trapezoidal_babd``.
"""
from __future__ import annotations

import collections
import math
import time
from dataclasses import dataclass, field

import torch

from . import (AbdPlan, BT_STATUS, _lib, abd_factor, abd_plan_destroy, abd_solve, bt_plan_create_in,
               bt_plan_workspace_size, bt_refine_async, bt_refine_result)


@dataclass
class BvpSpec:
    """Compact description of one BVP: L(t) = S + cos(2 pi t) K, boundary
    blocks B0, B1 (host float64 arrays, m x m)."""
    S: object
    K: object
    B0: object
    B1: object


@dataclass
class Request:
    rid: int
    arrival: float             # seconds since the start of the trace
    problem_id: int            # equal ids share (S, K, B0, B1, N): factorization reuse
    spec: BvpSpec
    N: int
    V: object                  # host [m, nrhs] float64
    prec: str = "fp64"
    # filled by the server
    t_admit: float = -1.0
    t_done: float = -1.0
    status: int = -1
    relcorr: float = 0.0
    cache_hit: bool = False
    fallback: bool = False     # refined path did not converge: solved again in FP64
    Y: object = None           # device solution [(N+1)*m, nrhs]
    Yexact_err: float = float("nan")

    @property
    def m(self):
        return self.spec.S.shape[0]

    @property
    def nrhs(self):
        return self.V.shape[1]

    @property
    def latency(self):
        return self.t_done - self.arrival


def build_bvp_device(spec: BvpSpec, N: int, device, stream=None):
    """(S_j, R_j, B0, B1) of the trapezoidal rule on t_j = j/N, on the device,
    built in place (no L(t) array): S_j = -(I + h/2 L(t_j)), R_j = I - h/2 L(t_{j+1})."""
    m = spec.S.shape[0]
    h = 1.0 / N
    with torch.cuda.stream(stream) if stream is not None else _nullctx():
        S0 = torch.as_tensor(spec.S, dtype=torch.float64, device=device)
        K = torch.as_tensor(spec.K, dtype=torch.float64, device=device)
        eye = torch.eye(m, dtype=torch.float64, device=device)
        t = torch.arange(N + 1, dtype=torch.float64, device=device) * h
        c = torch.cos(2 * math.pi * t).view(-1, 1, 1)
        Smat = c[:-1] * K.unsqueeze(0)                      # cos(2 pi t_j) K
        Smat.add_(S0).mul_(-0.5 * h).sub_(eye)
        Rmat = c[1:] * K.unsqueeze(0)
        Rmat.add_(S0).mul_(-0.5 * h).add_(eye)
        B0 = torch.as_tensor(spec.B0, dtype=torch.float64, device=device)
        B1 = torch.as_tensor(spec.B1, dtype=torch.float64, device=device)
        return Smat.contiguous(), Rmat.contiguous(), B0.contiguous(), B1.contiguous()


def build_rhs_device(spec: BvpSpec, N: int, V, device, stream=None):
    """Right-hand side [(N+1)*m, nrhs] (boundary row first) for the exact
    solution y(t) = exp(sin 3t) v, and that exact solution on the grid."""
    m = spec.S.shape[0]
    h = 1.0 / N
    with torch.cuda.stream(stream) if stream is not None else _nullctx():
        S0 = torch.as_tensor(spec.S, dtype=torch.float64, device=device)
        K = torch.as_tensor(spec.K, dtype=torch.float64, device=device)
        Vd = torch.as_tensor(V, dtype=torch.float64, device=device)
        t = torch.arange(N + 1, dtype=torch.float64, device=device) * h
        e = torch.exp(torch.sin(3 * t)).view(-1, 1, 1)
        SV, KV = S0 @ Vd, K @ Vd                                   # L(t) y = e (S0 v + cos K v)
        q = (3 * torch.cos(3 * t)).view(-1, 1, 1) * Vd.unsqueeze(0)
        q.sub_(SV.unsqueeze(0)).sub_(torch.cos(2 * math.pi * t).view(-1, 1, 1) * KV.unsqueeze(0)).mul_(e)
        r = (q[:-1] + q[1:]).mul_(0.5 * h)
        B0 = torch.as_tensor(spec.B0, dtype=torch.float64, device=device)
        B1 = torch.as_tensor(spec.B1, dtype=torch.float64, device=device)
        y0, yN = Vd, math.exp(math.sin(3.0)) * Vd
        beta = B0 @ y0 + B1 @ yN
        rhs = torch.cat([beta.unsqueeze(0), r], dim=0).reshape((N + 1) * m, -1).contiguous()
        yex = (e * Vd.unsqueeze(0)).reshape((N + 1) * m, -1)
        return rhs, yex


class _nullctx:
    def __enter__(self):
        return self

    def __exit__(self, *a):
        return False


def _round_nrhs(n):
    for c in (1, 4, 8, 16, 32):
        if n <= c:
            return c
    raise ValueError("at most 32 right-hand sides")


class _Factor:
    """A cached factorization: plan on pooled workspace + its matrices."""

    def __init__(self, key, plan, ws, mats, nrhs_max, nbytes, stream):
        self.key, self.plan, self.ws, self.mats = key, plan, ws, mats
        self.nrhs_max, self.nbytes, self.stream = nrhs_max, nbytes, stream
        self.busy = 0
        self.ready_event = None

    def destroy(self):
        if self.plan is not None:
            abd_plan_destroy(self.plan)
            self.plan = None
        self.ws = None
        self.mats = None


class Server:
    def __init__(self, device=None, mem_cap_bytes: float = 150e9, streams: int = 8, sweeps: int = 3,
                 tol: float = 1e-12, cache: bool = True, check_exact: bool = False, max_inflight: int = 0,
                 keep_results: bool = True, fp64_fallback: bool = True):
        self.device = torch.device(device or "cuda")
        self.cap = int(mem_cap_bytes)
        self.streams = [torch.cuda.Stream(device=self.device) for _ in range(streams)]
        self.sweeps = sweeps
        self.tol = tol
        self.cache_enabled = cache
        self.check_exact = check_exact
        self.queue = collections.deque()
        self.running = []            # (request, event, factor, transient bytes)
        self.done = []
        self.cache = collections.OrderedDict()   # key -> _Factor
        self.in_use = 0              # bytes of running requests + cached factors
        self.t0 = None
        self._next_stream = 0
        self.max_inflight = max_inflight if max_inflight > 0 else 2 * streams
        self.keep_results = keep_results
        # a refined request whose fixed sweeps end above the backward-error test
        # (BT_ERR_NOT_CONVERGED) is queued again, first, as an FP64 request
        self.fp64_fallback = fp64_fallback
        self._not_converged = next(k for k, v in BT_STATUS.items() if v == "BT_ERR_NOT_CONVERGED")
        total = torch.cuda.get_device_properties(self.device).total_memory
        self.cap = min(self.cap, int(0.7 * total))      # headroom for the caching allocator
        self.peak_in_use = 0
        _lib.load()

    # ------------------------------------------------------------ helpers --
    def now(self):
        return time.perf_counter() - self.t0

    def _key(self, r: Request):
        return (r.problem_id, r.N, r.m, r.prec)

    def footprint(self, r: Request) -> int:
        """Device bytes a request needs while it runs (plan workspace, matrices, vectors)."""
        ws, mats, vecs = self._footprint(r, _round_nrhs(r.nrhs))
        return ws + mats + vecs

    def _footprint(self, r: Request, nrhs_max):
        m, N = r.m, r.N
        ws = bt_plan_workspace_size(1, N, m, nrhs_max, r.prec)
        mats = 2 * N * m * m * 8 + 2 * m * m * 8
        vecs = 6 * (N + 1) * m * r.nrhs * 8 + (N + 1) * m * m * 8   # rhs, solution, exact, build temporaries
        return ws, mats, vecs

    def _evict_for(self, need, keep=None):
        """Release idle cached factorizations (least recently used first) until
        need bytes fit; never the one under `keep`, which the caller reuses."""
        for key in list(self.cache.keys()):
            if self.in_use + need <= self.cap:
                break
            if key == keep:
                continue
            f = self.cache[key]
            if f.busy == 0:
                f.destroy()
                self.in_use -= f.nbytes
                del self.cache[key]
        return self.in_use + need <= self.cap

    # ---------------------------------------------------------- interface --
    def start(self):
        self.t0 = time.perf_counter()

    def submit(self, r: Request):
        if self.t0 is None:
            self.start()
        self.queue.append(r)

    def _launch(self, r: Request) -> bool:
        key = self._key(r)
        f = self.cache.get(key) if self.cache_enabled else None
        if f is not None and f.busy and r.prec != "fp64":
            # the refinement's norms live in the plan: one refined request per plan at a time
            return False
        if f is not None and f.nrhs_max < r.nrhs:
            f = None if f.busy else f
            if f is not None:
                f.destroy()
                self.in_use -= f.nbytes
                del self.cache[key]
                f = None
        ws_b, mat_b, vec_b = self._footprint(r, _round_nrhs(r.nrhs))
        need = vec_b + (0 if f is not None else ws_b + mat_b)
        if f is not None and self.in_use + need > self.cap and not self._evict_for(need, keep=key):
            if f.busy:
                return False        # requests in flight will release memory
            # only the reused factorization itself is in the way: give up the reuse
            f.destroy()
            self.in_use -= f.nbytes
            del self.cache[key]
            f = None
            need = vec_b + ws_b + mat_b
        if need > self.cap:
            # can never fit: fail it now instead of holding the queue
            r.status = 2            # BT_ERR_NOMEM
            r.t_admit = r.t_done = self.now()
            r.Y = None
            self.done.append(r)
            return True
        if self.in_use + need > self.cap and not self._evict_for(need, keep=key if f is not None else None):
            return False
        if f is not None:
            r.cache_hit = True
            self.cache.move_to_end(key)
            stream = f.stream
        else:
            stream = self.streams[self._next_stream % len(self.streams)]
            self._next_stream += 1
        r.t_admit = self.now()
        with torch.cuda.stream(stream):
            if f is None:
                nr_max = _round_nrhs(r.nrhs)
                mats = build_bvp_device(r.spec, r.N, self.device, stream)
                ws = torch.empty(ws_b + 256, dtype=torch.uint8, device=self.device)
                off = (-ws.data_ptr()) % 256
                plan = bt_plan_create_in(1, r.N, r.m, nr_max, r.prec, ws.data_ptr() + off, ws_b, None,
                                         stream.cuda_stream)
                abd_factor(plan, *mats)
                f = _Factor(key, plan, ws, mats, nr_max, ws_b + mat_b, stream)
                self.in_use += f.nbytes
                if self.cache_enabled:
                    self.cache[key] = f
            f.busy += 1
            rhs, yex = build_rhs_device(r.spec, r.N, r.V, self.device, stream)
            Y = torch.empty_like(rhs)
            if r.prec == "fp64":
                abd_solve(f.plan, rhs, Y, r.nrhs)
            else:
                bt_refine_async(f.plan, rhs, Y, r.nrhs, self.sweeps)
            if self.check_exact:
                r.Yexact_err = (Y - yex).abs().max()
            ev = torch.cuda.Event()
            ev.record(stream)
        r.Y = Y
        self.in_use += vec_b
        self.running.append((r, ev, f, vec_b, rhs, yex))
        return True

    def poll(self):
        """Retire finished requests, then admit queued ones (in arrival order)."""
        still = []
        retry = []
        for item in self.running:
            r, ev, f, vec_b, rhs, yex = item
            if ev.query():
                r.t_done = self.now()
                if r.prec == "fp64":
                    r.status = _lib.load().abd_sync(f.plan)
                else:
                    r.status, r.relcorr = bt_refine_result(f.plan, self.tol)
                if self.check_exact and torch.is_tensor(r.Yexact_err):
                    r.Yexact_err = float(r.Yexact_err)
                if not self.keep_results:
                    r.Y = None
                f.busy -= 1
                self.in_use -= vec_b
                if self.cache.get(f.key) is not f:
                    if f.busy == 0:
                        f.destroy()
                        self.in_use -= f.nbytes
                if r.prec != "fp64" and r.status == self._not_converged and self.fp64_fallback:
                    r.fallback = True
                    r.prec = "fp64"
                    r.status, r.relcorr, r.Y, r.cache_hit = -1, 0.0, None, False
                    retry.append(r)
                else:
                    self.done.append(r)
            else:
                still.append(item)
        self.running = still
        for r in reversed(retry):
            self.queue.appendleft(r)
        while self.queue and len(self.running) < self.max_inflight:
            if not self._launch(self.queue[0]):
                break
            self.queue.popleft()
            self.peak_in_use = max(self.peak_in_use, self.in_use)

    def drain(self, timeout_s: float = 600.0):
        t_end = time.perf_counter() + timeout_s
        while (self.queue or self.running) and time.perf_counter() < t_end:
            self.poll()
            if self.running:
                time.sleep(0.0002)
        if self.queue or self.running:
            raise TimeoutError("server did not drain")

    def close(self):
        torch.cuda.synchronize(self.device)
        for f in self.cache.values():
            f.destroy()
        self.cache.clear()

    # -------------------------------------------------------------- trace --
    def run_trace(self, requests, realtime: bool = True, timeout_s: float = 900.0, keep_results: bool = False):
        """Replay requests at their arrival times (or all at once).  Solutions
        are dropped at retirement unless keep_results."""
        self.keep_results = keep_results
        self.start()
        pending = sorted(requests, key=lambda r: r.arrival)
        k = 0
        t_end = time.perf_counter() + timeout_s
        while (k < len(pending) or self.queue or self.running) and time.perf_counter() < t_end:
            now = self.now()
            while k < len(pending) and (not realtime or pending[k].arrival <= now):
                self.queue.append(pending[k])
                k += 1
            self.poll()
            time.sleep(0.0001)
        if k < len(pending) or self.queue or self.running:
            raise TimeoutError("trace did not finish")
        return self.stats()

    def stats(self):
        lat = sorted(r.latency for r in self.done)
        if not lat:
            return {}
        pct = lambda q: lat[min(len(lat) - 1, int(q * len(lat)))]   # noqa: E731
        span = max(r.t_done for r in self.done) - min(r.arrival for r in self.done)
        unk = sum((r.N + 1) * r.m * r.nrhs for r in self.done)
        return {"requests": len(self.done), "p50_ms": 1e3 * pct(0.50), "p99_ms": 1e3 * pct(0.99),
                "mean_ms": 1e3 * sum(lat) / len(lat), "span_s": span,
                "unknowns_per_s": unk / span if span > 0 else float("nan"),
                "cache_hits": sum(r.cache_hit for r in self.done),
                "fp64_fallbacks": sum(r.fallback for r in self.done),
                "failed": sum(r.status != 0 for r in self.done)}


def requests_from_trace(trace, prec="fp64"):
    """Requests of a ``gen.serve_trace`` trace (problem descriptions seeded by problem id)."""
    import numpy as np

    import gen
    out = []
    specs = {}
    for k, tr in enumerate(trace):
        if tr.problem_id not in specs:
            prng = np.random.Generator(np.random.PCG64(gen.SEED_BASE + 5000 * 1000 + 7919 * (tr.problem_id + 1)))
            p = gen.bvp_problem(tr.m, 1, rng=prng)
            specs[tr.problem_id] = BvpSpec(p.Smat, p.K, p.B0, p.B1)
        vrng = np.random.Generator(np.random.PCG64(tr.v_seed))
        V = vrng.standard_normal((tr.m, tr.nrhs))
        out.append(Request(k, tr.arrival_s, tr.problem_id, specs[tr.problem_id], tr.N, V, prec))
    return out
