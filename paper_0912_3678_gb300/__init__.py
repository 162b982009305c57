"""GB300 partition-method solver for structured sparse systems A x = f
(Amodio & Brugnano, "Parallel Factorizations in Numerical Analysis").

A thin binding over the C ABI of ``include/bt.h``: the functions below have
the C names and only marshal arguments (torch CUDA tensors -> device
pointers, the current torch stream -> cudaStream_t).  Every step of the
solve runs in the CUDA kernels of ``libbt.so``.  ``BtPlan``/``AbdPlan`` wrap
a plan handle with the same calls as methods.
"""
from __future__ import annotations

import ctypes

from . import _lib
from ._lib import BT_STATUS, PREC, BtBatchDesc, BtError, BtTuning

__all__ = ["BtPlan", "AbdPlan", "PbtPlan", "BtError", "BT_STATUS", "PREC", "load_library",
           "bt_plan_create", "bt_factor", "bt_solve", "bt_residual", "bt_refine_residual", "abd_refine_residual",
           "bt_refine", "bt_sync", "bt_info",
           "bt_plan_levels", "bt_plan_bytes", "bt_plan_trace", "bt_plan_trace_query", "bt_plan_launches",
           "KERNEL_KINDS", "bt_solve_noalloc", "BT_NOALLOC_SCRATCH_BYTES", "bt_plan_create_tuned",
           "bt_batch_create", "bt_batch_run", "bt_batch_finish", "bt_batch_info", "bt_batch_destroy",
           "BtBatch", "CycPlan", "cyc_plan_create", "cyc_factor", "cyc_solve", "cyc_residual", "cyc_refine",
           "BtTuning", "BtBatchDesc", "bt_refine_async", "bt_refine_result",
           "bt_plan_workspace_size", "bt_plan_anorm", "bt_plan_set_pivot_tol", "bt_plan_set_backward_tol", "bt_plan_set_forward_tol", "ivp_parareal", "ivp_bvm", "bt_plan_create_in", "bt_plan_capture", "bt_plan_replay", "bt_factor_solve_host", "bt_plan_capture_host",
           "abd_plan_create_tuned",
           "bt_band_to_blocks", "band_to_blocks", "bt_device_rcp", "bt_reduced_export", "bt_plan_destroy", "bt_status_string",
           "abd_plan_create", "abd_factor", "abd_solve", "abd_residual", "abd_refine", "abd_sync",
           "abd_plan_destroy"]


def load_library():
    return _lib.load()


def _ptr(t):
    if t is None:
        return None
    if isinstance(t, int):
        return t
    import torch
    if not isinstance(t, torch.Tensor):
        raise TypeError("expected a torch.Tensor or an int device pointer")
    if not t.is_cuda or t.dtype != torch.float64 or not t.is_contiguous():
        raise ValueError("arrays must be contiguous float64 CUDA tensors")
    return t.data_ptr()


def _stream(stream):
    if stream is None:
        import torch
        return torch.cuda.current_stream().cuda_stream
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream


def _prec(prec):
    return PREC[prec] if isinstance(prec, str) else int(prec)


# ---------------------------------------------------------------- C names --

def bt_status_string(code: int) -> str:
    return _lib.load().bt_status_string(code).decode()


def bt_plan_create(nblk, m, nrhs_max=1, prec="fp64", p=0, stream=None):
    h = ctypes.c_void_p()
    _lib.check(_lib.load().bt_plan_create(ctypes.byref(h), int(nblk), int(m), int(nrhs_max), _prec(prec),
                                          int(p), _stream(stream)), "bt_plan_create")
    return h


def _tuning(t):
    if t is None:
        return None
    if isinstance(t, BtTuning):
        return t
    return BtTuning(int(t.get("p0", 0)), int(t.get("ctas_per_sm", 0)), int(t.get("sub_rows", 0)),
                    int(t.get("top_rows", 0)), int(t.get("reduced", 0)), int(t.get("tp_block", 0)),
                    int(t.get("local", 0)), int(t.get("pivot", 0)), int(t.get("serial", 0)))


def bt_plan_create_tuned(nblk, m, nrhs_max=1, prec="fp64", tuning=None, stream=None):
    h = ctypes.c_void_p()
    t = _tuning(tuning)
    _lib.check(_lib.load().bt_plan_create_tuned(ctypes.byref(h), int(nblk), int(m), int(nrhs_max), _prec(prec),
                                                ctypes.byref(t) if t is not None else None, _stream(stream)),
               "bt_plan_create_tuned")
    return h


def bt_batch_create(descs, ir_sweeps=3, mem_cap_bytes=0, stream=None):
    arr = (BtBatchDesc * len(descs))(*descs)
    h = ctypes.c_void_p()
    _lib.check(_lib.load().bt_batch_create(ctypes.byref(h), arr, len(descs), int(ir_sweeps), int(mem_cap_bytes),
                                           _stream(stream)), "bt_batch_create")
    return h


def bt_batch_run(batch):
    _lib.check(_lib.load().bt_batch_run(batch), "bt_batch_run")


def bt_batch_finish(batch, count, tol=1e-12):
    st = (ctypes.c_int * count)()
    rc = (ctypes.c_double * count)()
    code = _lib.load().bt_batch_finish(batch, float(tol), st, rc)
    return code, list(st), list(rc)


def bt_batch_info(batch):
    w = ctypes.c_int(0)
    n = ctypes.c_int64(0)
    b = ctypes.c_int64(0)
    _lib.check(_lib.load().bt_batch_info(batch, ctypes.byref(w), ctypes.byref(n), ctypes.byref(b)),
               "bt_batch_info")
    return w.value, n.value, b.value


def bt_batch_destroy(batch):
    _lib.load().bt_batch_destroy(batch)


def abd_plan_create(N, m, nrhs_max=1, prec="fp64", p=0, stream=None):
    h = ctypes.c_void_p()
    _lib.check(_lib.load().abd_plan_create(ctypes.byref(h), int(N), int(m), int(nrhs_max), _prec(prec),
                                           int(p), _stream(stream)), "abd_plan_create")
    return h


def abd_plan_create_tuned(N, m, nrhs_max=1, prec="fp64", tuning=None, stream=None):
    h = ctypes.c_void_p()
    t = _tuning(tuning)
    _lib.check(_lib.load().abd_plan_create_tuned(ctypes.byref(h), int(N), int(m), int(nrhs_max), _prec(prec),
                                                 ctypes.byref(t) if t is not None else None, _stream(stream)),
               "abd_plan_create_tuned")
    return h


def bt_factor(plan, B, D, C):
    _lib.check(_lib.load().bt_factor(plan, _ptr(B), _ptr(D), _ptr(C)), "bt_factor")


def abd_factor(plan, S, R, B0, B1):
    _lib.check(_lib.load().abd_factor(plan, _ptr(S), _ptr(R), _ptr(B0), _ptr(B1)), "abd_factor")


def bt_solve(plan, F, X, nrhs):
    _lib.check(_lib.load().bt_solve(plan, _ptr(F), _ptr(X), int(nrhs)), "bt_solve")


def abd_solve(plan, RHS, Y, nrhs):
    _lib.check(_lib.load().abd_solve(plan, _ptr(RHS), _ptr(Y), int(nrhs)), "abd_solve")


def bt_residual(plan, F, X, R, nrhs):
    _lib.check(_lib.load().bt_residual(plan, _ptr(F), _ptr(X), _ptr(R), int(nrhs)), "bt_residual")


def abd_residual(plan, RHS, Y, Rout, nrhs):
    _lib.check(_lib.load().abd_residual(plan, _ptr(RHS), _ptr(Y), _ptr(Rout), int(nrhs)), "abd_residual")


def bt_refine_residual(plan, F, X, R, nrhs):
    """The residual as the plan's refinement forms it (FP64-accurate, rounded to FP32 precision)."""
    _lib.check(_lib.load().bt_refine_residual(plan, _ptr(F), _ptr(X), _ptr(R), int(nrhs)), "bt_refine_residual")


def abd_refine_residual(plan, RHS, Y, Rout, nrhs):
    _lib.check(_lib.load().abd_refine_residual(plan, _ptr(RHS), _ptr(Y), _ptr(Rout), int(nrhs)),
               "abd_refine_residual")


def _refine(fn, name, plan, F, X, nrhs, tol, maxit, raise_on_error):
    it = ctypes.c_int(0)
    rc = ctypes.c_double(0.0)
    code = fn(plan, _ptr(F), _ptr(X), int(nrhs), float(tol), int(maxit), ctypes.byref(it), ctypes.byref(rc))
    if raise_on_error:
        _lib.check(code, name)
    return code, it.value, rc.value


def bt_refine(plan, F, X, nrhs, tol=1e-12, maxit=30, raise_on_error=True):
    return _refine(_lib.load().bt_refine, "bt_refine", plan, F, X, nrhs, tol, maxit, raise_on_error)


def abd_refine(plan, RHS, Y, nrhs, tol=1e-12, maxit=30, raise_on_error=True):
    return _refine(_lib.load().abd_refine, "abd_refine", plan, RHS, Y, nrhs, tol, maxit, raise_on_error)


def cyc_plan_create(N, m, nrhs_max=1, prec="fp64", p=0, stream=None):
    h = ctypes.c_void_p()
    _lib.check(_lib.load().cyc_plan_create(ctypes.byref(h), int(N), int(m), int(nrhs_max), _prec(prec),
                                           int(p), _stream(stream)), "cyc_plan_create")
    return h


def cyc_factor(plan, S, R):
    _lib.check(_lib.load().cyc_factor(plan, _ptr(S), _ptr(R)), "cyc_factor")


def cyc_solve(plan, RHS, Y, nrhs):
    _lib.check(_lib.load().cyc_solve(plan, _ptr(RHS), _ptr(Y), int(nrhs)), "cyc_solve")


def cyc_residual(plan, RHS, Y, Rout, nrhs):
    _lib.check(_lib.load().cyc_residual(plan, _ptr(RHS), _ptr(Y), _ptr(Rout), int(nrhs)), "cyc_residual")


def cyc_refine(plan, RHS, Y, nrhs, tol=1e-12, maxit=30, raise_on_error=True):
    return _refine(_lib.load().cyc_refine, "cyc_refine", plan, RHS, Y, nrhs, tol, maxit, raise_on_error)


def bt_refine_async(plan, F, X, nrhs, sweeps=2):
    _lib.check(_lib.load().bt_refine_async(plan, _ptr(F), _ptr(X), int(nrhs), int(sweeps)), "bt_refine_async")


def bt_refine_result(plan, tol=1e-12):
    rc = ctypes.c_double(0.0)
    code = _lib.load().bt_refine_result(plan, float(tol), ctypes.byref(rc))
    return code, rc.value


def ivp_parareal(dl, d, du, g0, y0, T, p, nfine, ncoarse=1, kmax=None, tol=1e-12, g1=None, U=None,
                 keep_history=False, stream=None, raise_on_error=True):
    """Parareal for y' = L y + g0 + t g1 (L tridiagonal: dl, d, du; CUDA float64
    vectors of length n) on [0, T] with p coarse intervals (see bt_ivp.h).
    Returns (U [p+1, n], iterations, status code, history [(kmax+1), p+1, n] or None)."""
    import torch
    n = d.shape[0]
    kmax = p if kmax is None else kmax
    U = torch.empty((p + 1, n), dtype=torch.float64, device=d.device) if U is None else U
    hist = torch.empty((kmax + 1, p + 1, n), dtype=torch.float64, device=d.device) if keep_history else None
    it = ctypes.c_int(0)
    code = _lib.load().ivp_parareal(int(n), _ptr(dl), _ptr(d), _ptr(du), _ptr(g0), _ptr(g1), _ptr(y0), float(T),
                                    int(p), int(nfine), int(ncoarse), int(kmax), float(tol), _ptr(U), _ptr(hist),
                                    ctypes.byref(it), _stream(stream))
    if raise_on_error and code not in (0, 5):
        _lib.check(code, "ivp_parareal")
    return U, it.value, code, hist


def ivp_bvm(L, y0, G, T, p, N, Y=None, stream=None):
    """Parallel IVP solver with the order-3 block BVM (see bt_ivp.h) for
    y' = L y + g(t): L [m, m], y0 [m], G [p N + 1, m] = g on the fine grid
    (CUDA float64).  Returns Y [p N + 1, m], Y[k] ~ y(k T / (p N))."""
    import torch
    m = L.shape[0]
    Y = torch.empty((p * N + 1, m), dtype=torch.float64, device=L.device) if Y is None else Y
    _lib.check(_lib.load().ivp_bvm(int(m), int(p), int(N), float(T), _ptr(L), _ptr(y0), _ptr(G), _ptr(Y),
                                   _stream(stream)), "ivp_bvm")
    return Y


class PbtPlan:
    """Block tridiagonal matrix with corner blocks (pbt_*, bt_pbt.h): B[0] couples
    row 0 to x_{N-1}, C[N-1] couples row N-1 to x_0; FP64."""

    def __init__(self, N, m, nrhs_max=1, p=0, stream=None):
        self.n, self.m, self.nrhs_max = int(N), int(m), int(nrhs_max)
        h = ctypes.c_void_p()
        _lib.check(_lib.load().pbt_plan_create(ctypes.byref(h), int(N), int(m), int(nrhs_max), int(p),
                                               _stream(stream)), "pbt_plan_create")
        self.handle = h
        self._keep = ()

    def factor(self, B, D, C):
        self._keep = (B, D, C)
        _lib.check(_lib.load().pbt_factor(self.handle, _ptr(B), _ptr(D), _ptr(C)), "pbt_factor")

    def solve(self, F, X=None):
        import torch
        X = torch.empty_like(F) if X is None else X
        nr = F.shape[1] if F.dim() == 2 else 1
        _lib.check(_lib.load().pbt_solve(self.handle, _ptr(F), _ptr(X), int(nr)), "pbt_solve")
        return X

    def residual(self, F, X, R=None):
        import torch
        R = torch.empty_like(F) if R is None else R
        nr = F.shape[1] if F.dim() == 2 else 1
        _lib.check(_lib.load().pbt_residual(self.handle, _ptr(F), _ptr(X), _ptr(R), int(nr)), "pbt_residual")
        return R

    def sync(self):
        _lib.check(_lib.load().pbt_sync(self.handle), "pbt_sync")

    def close(self):
        if getattr(self, "handle", None) is not None:
            _lib.load().pbt_plan_destroy(self.handle)
            self.handle = None

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def bt_plan_set_pivot_tol(plan, tau: float):
    _lib.check(_lib.load().bt_plan_set_pivot_tol(plan, float(tau)), "bt_plan_set_pivot_tol")


def bt_plan_set_backward_tol(plan, eta_tol: float):
    _lib.check(_lib.load().bt_plan_set_backward_tol(plan, float(eta_tol)), "bt_plan_set_backward_tol")


def bt_plan_set_forward_tol(plan, fwd_tol: float):
    """Estimated forward-error target of the refinement stopping test (<= 0: off)."""
    _lib.check(_lib.load().bt_plan_set_forward_tol(plan, float(fwd_tol)), "bt_plan_set_forward_tol")


def bt_plan_anorm(plan) -> float:
    """||A||_inf of the factored matrices as the refinement stopping test uses it."""
    v = ctypes.c_double(0.0)
    _lib.check(_lib.load().bt_plan_anorm(plan, ctypes.byref(v)), "bt_plan_anorm")
    return v.value


def bt_plan_workspace_size(kind, n, m, nrhs_max=1, prec="fp64", tuning=None) -> int:
    b = ctypes.c_int64(0)
    t = _tuning(tuning)
    _lib.check(_lib.load().bt_plan_workspace_size(int(kind), int(n), int(m), int(nrhs_max), _prec(prec),
                                                  ctypes.byref(t) if t is not None else None, ctypes.byref(b)),
               "bt_plan_workspace_size")
    return b.value


def bt_plan_create_in(kind, n, m, nrhs_max, prec, workspace, nbytes, tuning=None, stream=None):
    h = ctypes.c_void_p()
    t = _tuning(tuning)
    _lib.check(_lib.load().bt_plan_create_in(ctypes.byref(h), int(kind), int(n), int(m), int(nrhs_max),
                                             _prec(prec), ctypes.byref(t) if t is not None else None,
                                             _ptr_any(workspace), int(nbytes), _stream(stream)),
               "bt_plan_create_in")
    return h


def _ptr_any(t):
    return t if isinstance(t, int) else t.data_ptr()


CAPTURE = {"factor_solve": 1, "solve": 2, "factor_refine": 3}


def bt_plan_capture(plan, what, F, X, nrhs, sweeps=0):
    w = CAPTURE[what] if isinstance(what, str) else int(what)
    _lib.check(_lib.load().bt_plan_capture(plan, w, _ptr(F), _ptr(X), int(nrhs), int(sweeps)), "bt_plan_capture")


def bt_device_rcp(x, y=None, stream=None):
    """y = 1/x elementwise with the device FP64 reciprocal of the pivot steps."""
    import torch
    if y is None:
        y = torch.empty_like(x)
    _lib.check(_lib.load().bt_device_rcp(int(x.numel()), _ptr(x), _ptr(y), _stream(stream)), "bt_device_rcp")
    return y


def bt_band_to_blocks(n, s, r, band, m, B, D, C, stream=None):
    _lib.check(_lib.load().bt_band_to_blocks(int(n), int(s), int(r), _ptr(band), int(m), _ptr(B), _ptr(D),
                                             _ptr(C), _stream(stream)), "bt_band_to_blocks")


def band_to_blocks(band, s, r, m=None):
    """Banded matrix (band storage [s + r + 1, n] CUDA float64 tensor) -> block
    tridiagonal (B, D, C) of order m = max(s, r, 1) (or the given m)."""
    import torch
    n = band.shape[1]
    m = max(s, r, 1) if m is None else m
    N = (n + m - 1) // m
    B = torch.empty((N, m, m), dtype=torch.float64, device=band.device)
    D = torch.empty_like(B)
    C = torch.empty_like(B)
    bt_band_to_blocks(n, s, r, band, m, B, D, C)
    return B, D, C


def _host_ptr(t):
    """Address of a host float64 array (a CPU torch tensor, pinned or not, or a numpy array)."""
    import numpy as np
    import torch
    if isinstance(t, torch.Tensor):
        if t.is_cuda or t.dtype != torch.float64 or not t.is_contiguous():
            raise TypeError("expected a contiguous CPU float64 tensor")
        return t.data_ptr()
    if isinstance(t, np.ndarray):
        if t.dtype != np.float64 or not t.flags["C_CONTIGUOUS"]:
            raise TypeError("expected a C-contiguous float64 array")
        return t.ctypes.data
    raise TypeError("expected a host array")


def bt_factor_solve_host(plan, B, D, C, F, X, nrhs, sweeps=-1):
    """Factor + solve (or + `sweeps` refinement corrections) from host arrays (see bt.h)."""
    _lib.check(_lib.load().bt_factor_solve_host(plan, _host_ptr(B), _host_ptr(D), _host_ptr(C), _host_ptr(F),
                                                _host_ptr(X), int(nrhs), int(sweeps)), "bt_factor_solve_host")


def bt_plan_capture_host(plan, B, D, C, F, X, nrhs, sweeps=-1):
    """Record bt_factor_solve_host (pinned host arrays) into the plan's graph; replay() re-runs it."""
    _lib.check(_lib.load().bt_plan_capture_host(plan, _host_ptr(B), _host_ptr(D), _host_ptr(C), _host_ptr(F),
                                                _host_ptr(X), int(nrhs), int(sweeps)), "bt_plan_capture_host")


def bt_plan_replay(plan):
    _lib.check(_lib.load().bt_plan_replay(plan), "bt_plan_replay")


def bt_sync(plan) -> int:
    return _lib.load().bt_sync(plan)


def abd_sync(plan) -> int:
    return _lib.load().abd_sync(plan)


def bt_info(plan):
    lev = ctypes.c_int(0)
    part = ctypes.c_int64(0)
    row = ctypes.c_int64(0)
    code = _lib.load().bt_info(plan, ctypes.byref(lev), ctypes.byref(part), ctypes.byref(row))
    return code, lev.value, part.value, row.value


def bt_plan_levels(plan):
    n = ctypes.c_int(0)
    cap = 64
    rows = (ctypes.c_int64 * cap)()
    parts = (ctypes.c_int64 * cap)()
    _lib.check(_lib.load().bt_plan_levels(plan, ctypes.byref(n), rows, parts, cap), "bt_plan_levels")
    return [(rows[i], parts[i]) for i in range(min(n.value, cap))]


def bt_plan_bytes(plan) -> int:
    b = ctypes.c_int64(0)
    _lib.check(_lib.load().bt_plan_bytes(plan, ctypes.byref(b)), "bt_plan_bytes")
    return b.value


def bt_reduced_export(plan, alpha, beta, gamma=None):
    _lib.check(_lib.load().bt_reduced_export(plan, _ptr(alpha), _ptr(beta), _ptr(gamma)), "bt_reduced_export")


KERNEL_KINDS = {"factor": 0, "assemble": 1, "solve_fwd": 2, "assemble_rhs": 3, "solve_bwd": 4,
                "direct": 5, "residual": 6, "ir_update": 7, "bcr_factor": 8, "bcr_solve": 9,
                "norm": 10}


def bt_plan_trace(plan, enable=True):
    _lib.check(_lib.load().bt_plan_trace(plan, 1 if enable else 0), "bt_plan_trace")


def bt_plan_trace_query(plan, kind, level=-1):
    ms = ctypes.c_double(0.0)
    n = ctypes.c_int64(0)
    k = KERNEL_KINDS[kind] if isinstance(kind, str) else int(kind)
    _lib.check(_lib.load().bt_plan_trace_query(plan, k, int(level), ctypes.byref(ms), ctypes.byref(n)),
               "bt_plan_trace_query")
    return ms.value, n.value


def bt_plan_launches(plan) -> int:
    n = ctypes.c_int64(0)
    _lib.check(_lib.load().bt_plan_launches(plan, ctypes.byref(n)), "bt_plan_launches")
    return n.value


def bt_plan_destroy(plan):
    _lib.load().bt_plan_destroy(plan)


BT_NOALLOC_SCRATCH_BYTES = 8 << 20


def bt_solve_noalloc(nblk, m, B, D, C, F, X, nrhs, stream=None):
    """One-shot FP64 solve with no device allocation (see include/bt.h).
    Returns (status code, required scratch bytes); does not raise."""
    req = ctypes.c_int64(0)
    code = _lib.load().bt_solve_noalloc(int(nblk), int(m), _ptr(B), _ptr(D), _ptr(C), _ptr(F), _ptr(X),
                                        int(nrhs), _stream(stream), ctypes.byref(req))
    return code, req.value


def abd_plan_destroy(plan):
    _lib.load().abd_plan_destroy(plan)


# ---------------------------------------------------------------- classes --

class _PlanBase:
    kind = 0

    def __init__(self, n, m, nrhs_max=1, prec="fp64", p=0, stream=None):
        import torch
        self.m = int(m)
        self.n = int(n)
        self.nrhs_max = int(nrhs_max)
        self.prec = prec
        self.stream = stream
        self.rows = self.n if self.kind == 0 else self.n + 1
        create = bt_plan_create if self.kind == 0 else abd_plan_create
        self.handle = create(n, m, nrhs_max, prec, p, stream)
        self._keep = ()
        self._torch = torch

    def _new_like_rhs(self, F):
        return self._torch.empty_like(F)

    def _nrhs(self, F):
        return 1 if F.dim() == 1 else F.shape[-1]

    def close(self):
        if getattr(self, "handle", None) is not None:
            (bt_plan_destroy if self.kind == 0 else abd_plan_destroy)(self.handle)
            self.handle = None
            self._keep = ()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def sync(self):
        code = bt_sync(self.handle)
        _lib.check(code, "sync")

    def info(self):
        return bt_info(self.handle)

    def levels(self):
        return bt_plan_levels(self.handle)

    def nbytes(self):
        return bt_plan_bytes(self.handle)

    def trace(self, enable=True):
        bt_plan_trace(self.handle, enable)

    def trace_query(self, kind, level=-1):
        return bt_plan_trace_query(self.handle, kind, level)

    def launches(self):
        return bt_plan_launches(self.handle)

    def capture(self, what, F, X, sweeps=0):
        """Record factor/solve (see bt_plan_capture) into a CUDA graph; replay() re-runs it."""
        bt_plan_capture(self.handle, what, F, X, self._nrhs(F), sweeps)

    def replay(self):
        bt_plan_replay(self.handle)

    def factor_solve_host(self, B, D, C, F, X, sweeps=-1):
        """bt_factor_solve_host: host (pinned) B, D, C, F in, host X out, asynchronous."""
        nr = F.shape[1] if len(F.shape) == 2 else 1
        bt_factor_solve_host(self.handle, B, D, C, F, X, nr, sweeps)

    def capture_host(self, B, D, C, F, X, sweeps=-1):
        """bt_plan_capture_host: the host-array call as one graph; replay() re-runs it."""
        nr = F.shape[1] if len(F.shape) == 2 else 1
        bt_plan_capture_host(self.handle, B, D, C, F, X, nr, sweeps)

    def set_forward_tol(self, fwd_tol: float):
        """Estimated forward-error target of the refinement stopping test (<= 0: off)."""
        bt_plan_set_forward_tol(self.handle, fwd_tol)


class BtPlan(_PlanBase):
    """Block tridiagonal plan: B_j x_{j-1} + D_j x_j + C_j x_{j+1} = f_j."""
    kind = 0

    @classmethod
    def tuned(cls, nblk, m, nrhs_max=1, prec="fp64", tuning=None, stream=None):
        """A plan with explicit partitioning parameters (see tune.Tuner)."""
        import torch
        self = cls.__new__(cls)
        self.m, self.n, self.nrhs_max, self.prec, self.stream = int(m), int(nblk), int(nrhs_max), prec, stream
        self.rows = self.n
        self.handle = bt_plan_create_tuned(nblk, m, nrhs_max, prec, tuning, stream)
        self._local = int((tuning or {}).get("local", 0)) if isinstance(tuning, (dict, type(None))) else int(tuning.local)
        self._keep = ()
        self._torch = torch
        return self

    def factor(self, B, D, C):
        self._keep = (B, D, C)
        bt_factor(self.handle, B, D, C)

    def solve(self, F, X=None):
        X = self._new_like_rhs(F) if X is None else X
        bt_solve(self.handle, F, X, self._nrhs(F))
        return X

    def residual(self, F, X, R=None):
        R = self._new_like_rhs(F) if R is None else R
        bt_residual(self.handle, F, X, R, self._nrhs(F))
        return R

    def refine_residual(self, F, X, R=None):
        """bt_refine_residual: the residual the refinement uses."""
        R = self._new_like_rhs(F) if R is None else R
        bt_refine_residual(self.handle, F, X, R, self._nrhs(F))
        return R

    def refine(self, F, X=None, tol=1e-12, maxit=30, raise_on_error=True):
        X = self._new_like_rhs(F) if X is None else X
        code, it, rc = bt_refine(self.handle, F, X, self._nrhs(F), tol, maxit, raise_on_error)
        return X, it, rc, code

    def anorm(self) -> float:
        return bt_plan_anorm(self.handle)

    def reduced(self):
        """Top-level reduced matrix (alpha, beta, gamma) of Eq. (redmatr); with
        local cyclic reduction, the FP64 system on the separators."""
        lev = self.levels()
        q = lev[0][1] - 1
        if getattr(self, "_local", 0) > 0:
            steps, K = 0, self.n
            while K > 1:
                K, steps = (K + 1) // 2, steps + 1
            q = self.n
            for _ in range(min(self._local, steps)):
                q = (q + 1) // 2
        t = self._torch
        dev = self._keep[1].device
        a = t.empty((q, self.m, self.m), dtype=t.float64, device=dev)
        b = t.empty_like(a)
        g = t.empty_like(a)
        bt_reduced_export(self.handle, a, b, g)
        return a, b, g


class BtBatch:
    """Many independent block tridiagonal systems solved by one CUDA-graph
    launch.  ``systems``: list of dicts with keys B, D, C, F, X (CUDA float64
    tensors), prec ("fp64" | "fp32_ir" | "bf16_ir") and optional tuning."""

    def __init__(self, systems, ir_sweeps=3, mem_cap_bytes=0, stream=None, tuner=None):
        descs = []
        self._keep = []
        for sd in systems:
            D = sd["D"]
            N, m = D.shape[0], D.shape[1]
            F = sd["F"]
            nr = 1 if F.dim() == 1 else F.shape[-1]
            prec = sd.get("prec", "fp64")
            tun = sd.get("tuning")
            if tun is None and tuner is not None:
                tun = tuner(m, N, prec)
            descs.append(BtBatchDesc(N, m, _prec(prec), nr, _ptr(sd["B"]), _ptr(D), _ptr(sd["C"]), _ptr(F),
                                     _ptr(sd["X"]), _tuning(tun) or BtTuning(0, 0, 0, 0, 0, 0, 0, 0)))
            self._keep.append((sd["B"], D, sd["C"], F, sd["X"]))
        self.count = len(descs)
        self.handle = bt_batch_create(descs, ir_sweeps, mem_cap_bytes, stream)

    def run(self):
        bt_batch_run(self.handle)

    def finish(self, tol=1e-12):
        return bt_batch_finish(self.handle, self.count, tol)

    def info(self):
        return bt_batch_info(self.handle)

    def close(self):
        if getattr(self, "handle", None) is not None:
            bt_batch_destroy(self.handle)
            self.handle = None
            self._keep = []

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()


class CycPlan(_PlanBase):
    """Circulant-like plan: S_j y_j + R_j y_{(j+1) mod N} = r_j, j = 0..N-1
    (a BABD plan on the rows rotated by one)."""
    kind = 1

    def __init__(self, n, m, nrhs_max=1, prec="fp64", p=0, stream=None):
        import torch
        self.m, self.n, self.nrhs_max, self.prec, self.stream = int(m), int(n), int(nrhs_max), prec, stream
        self.rows = self.n
        self.handle = cyc_plan_create(n, m, nrhs_max, prec, p, stream)
        self._keep = ()
        self._torch = torch

    def factor(self, S, R):
        self._keep = (S, R)
        cyc_factor(self.handle, S, R)

    def solve(self, RHS, Y=None):
        Y = self._new_like_rhs(RHS) if Y is None else Y
        cyc_solve(self.handle, RHS, Y, self._nrhs(RHS))
        return Y

    def residual(self, RHS, Y, Rout=None):
        Rout = self._new_like_rhs(RHS) if Rout is None else Rout
        cyc_residual(self.handle, RHS, Y, Rout, self._nrhs(RHS))
        return Rout

    def refine(self, RHS, Y=None, tol=1e-12, maxit=30, raise_on_error=True):
        Y = self._new_like_rhs(RHS) if Y is None else Y
        code, it, rc = cyc_refine(self.handle, RHS, Y, self._nrhs(RHS), tol, maxit, raise_on_error)
        return Y, it, rc, code


class AbdPlan(_PlanBase):
    """BABD plan: B0 y_0 + B1 y_N = beta;  S_j y_j + R_j y_{j+1} = r_j."""
    kind = 1

    @classmethod
    def tuned(cls, N, m, nrhs_max=1, prec="fp64", tuning=None, stream=None):
        """A plan with explicit parameters; tuning {"reduced": 1}: cyclic reduction
        of the whole system (abd_plan_create_tuned)."""
        import torch
        self = cls.__new__(cls)
        self.m, self.n, self.nrhs_max, self.prec, self.stream = int(m), int(N), int(nrhs_max), prec, stream
        self.rows = self.n + 1
        self.handle = abd_plan_create_tuned(N, m, nrhs_max, prec, tuning, stream)
        self._keep = ()
        self._torch = torch
        return self

    def factor(self, S, R, B0, B1):
        self._keep = (S, R, B0, B1)
        abd_factor(self.handle, S, R, B0, B1)

    def solve(self, RHS, Y=None):
        Y = self._new_like_rhs(RHS) if Y is None else Y
        abd_solve(self.handle, RHS, Y, self._nrhs(RHS))
        return Y

    def residual(self, RHS, Y, Rout=None):
        Rout = self._new_like_rhs(RHS) if Rout is None else Rout
        abd_residual(self.handle, RHS, Y, Rout, self._nrhs(RHS))
        return Rout

    def refine_residual(self, RHS, Y, Rout=None):
        """abd_refine_residual: the residual the refinement uses."""
        Rout = self._new_like_rhs(RHS) if Rout is None else Rout
        abd_refine_residual(self.handle, RHS, Y, Rout, self._nrhs(RHS))
        return Rout

    def refine(self, RHS, Y=None, tol=1e-12, maxit=30, raise_on_error=True):
        Y = self._new_like_rhs(RHS) if Y is None else Y
        code, it, rc = abd_refine(self.handle, RHS, Y, self._nrhs(RHS), tol, maxit, raise_on_error)
        return Y, it, rc, code

    def anorm(self) -> float:
        return bt_plan_anorm(self.handle)

    def reduced(self):
        """Top-level reduced BABD matrix of Eq. (redmatr1): alpha [p+1], beta [p+1]
        (beta[0] is the corner block)."""
        lev = self.levels()
        q = lev[0][1] + 1
        t = self._torch
        dev = self._keep[0].device
        a = t.empty((q, self.m, self.m), dtype=t.float64, device=dev)
        b = t.empty_like(a)
        bt_reduced_export(self.handle, a, b, None)
        return a, b
