"""ctypes loader for ``_build/libbt.so`` (the C ABI of ``include/bt.h``).

There is no fallback: if the library is missing, importing the binding
raises, so nothing silently runs off the GPU path."""
from __future__ import annotations

import ctypes
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "_build", "libbt.so")

BT_STATUS = {
    0: "BT_OK", 1: "BT_ERR_INVALID", 2: "BT_ERR_NOMEM", 3: "BT_ERR_SINGULAR", 4: "BT_ERR_NONFINITE",
    5: "BT_ERR_NOT_CONVERGED", 6: "BT_ERR_TIMEOUT", 7: "BT_ERR_CUDA",
}
PREC = {"fp64": 0, "fp32_ir": 1, "bf16_ir": 2}

# name -> (restype, argtypes)
_vp, _i32, _i64, _f64 = ctypes.c_void_p, ctypes.c_int, ctypes.c_int64, ctypes.c_double
_pvp = ctypes.POINTER(ctypes.c_void_p)
_pi32 = ctypes.POINTER(ctypes.c_int)
_pi64 = ctypes.POINTER(ctypes.c_int64)
_pf64 = ctypes.POINTER(ctypes.c_double)
SIGNATURES = {
    "bt_status_string": (ctypes.c_char_p, [_i32]),
    "bt_plan_create": (_i32, [_pvp, _i64, _i32, _i32, _i32, _i64, _vp]),
    "bt_factor": (_i32, [_vp, _vp, _vp, _vp]),
    "bt_solve": (_i32, [_vp, _vp, _vp, _i32]),
    "bt_residual": (_i32, [_vp, _vp, _vp, _vp, _i32]),
    "bt_refine_residual": (_i32, [_vp, _vp, _vp, _vp, _i32]),
    "bt_refine": (_i32, [_vp, _vp, _vp, _i32, _f64, _i32, _pi32, _pf64]),
    "bt_sync": (_i32, [_vp]),
    "bt_info": (_i32, [_vp, _pi32, _pi64, _pi64]),
    "bt_plan_levels": (_i32, [_vp, _pi32, _pi64, _pi64, _i32]),
    "bt_plan_bytes": (_i32, [_vp, _pi64]),
    "bt_reduced_export": (_i32, [_vp, _vp, _vp, _vp]),
    "bt_plan_trace": (_i32, [_vp, _i32]),
    "bt_plan_trace_query": (_i32, [_vp, _i32, _i32, _pf64, _pi64]),
    "bt_plan_launches": (_i32, [_vp, _pi64]),
    "bt_plan_destroy": (None, [_vp]),
    "bt_solve_noalloc": (_i32, [_i64, _i32, _vp, _vp, _vp, _vp, _vp, _i32, _vp, _pi64]),
    "abd_plan_create": (_i32, [_pvp, _i64, _i32, _i32, _i32, _i64, _vp]),
    "abd_plan_create_tuned": (_i32, [_pvp, _i64, _i32, _i32, _i32, _vp, _vp]),
    "abd_factor": (_i32, [_vp, _vp, _vp, _vp, _vp]),
    "abd_solve": (_i32, [_vp, _vp, _vp, _i32]),
    "abd_residual": (_i32, [_vp, _vp, _vp, _vp, _i32]),
    "abd_refine_residual": (_i32, [_vp, _vp, _vp, _vp, _i32]),
    "abd_refine": (_i32, [_vp, _vp, _vp, _i32, _f64, _i32, _pi32, _pf64]),
    "abd_sync": (_i32, [_vp]),
    "abd_plan_destroy": (None, [_vp]),
}

class BtTuning(ctypes.Structure):
    _fields_ = [("p0", ctypes.c_int64), ("ctas_per_sm", ctypes.c_int), ("sub_rows", ctypes.c_int),
                ("top_rows", ctypes.c_int), ("reduced", ctypes.c_int), ("tp_block", ctypes.c_int),
                ("local", ctypes.c_int), ("pivot", ctypes.c_int),
                ("serial", ctypes.c_int)]


class BtBatchDesc(ctypes.Structure):
    _fields_ = [("nblk", ctypes.c_int64), ("m", ctypes.c_int), ("prec", ctypes.c_int), ("nrhs", ctypes.c_int),
                ("B", ctypes.c_void_p), ("D", ctypes.c_void_p), ("C", ctypes.c_void_p), ("F", ctypes.c_void_p),
                ("X", ctypes.c_void_p), ("tuning", BtTuning)]


SIGNATURES.update({
    "bt_plan_create_tuned": (_i32, [_pvp, _i64, _i32, _i32, _i32, ctypes.POINTER(BtTuning), _vp]),
    "bt_batch_create": (_i32, [_pvp, ctypes.POINTER(BtBatchDesc), _i32, _i32, _i64, _vp]),
    "bt_batch_run": (_i32, [_vp]),
    "bt_batch_finish": (_i32, [_vp, _f64, _pi32, _pf64]),
    "bt_batch_info": (_i32, [_vp, _pi32, _pi64, _pi64]),
    "bt_batch_destroy": (None, [_vp]),
    "bt_refine_async": (_i32, [_vp, _vp, _vp, _i32, _i32]),
    "bt_plan_capture": (_i32, [_vp, _i32, _vp, _vp, _i32, _i32]),
    "bt_plan_replay": (_i32, [_vp]),
    "bt_factor_solve_host": (_i32, [_vp, _vp, _vp, _vp, _vp, _vp, _i32, _i32]),
    "bt_plan_capture_host": (_i32, [_vp, _vp, _vp, _vp, _vp, _vp, _i32, _i32]),
    "bt_band_to_blocks": (_i32, [_i64, _i32, _i32, _vp, _i32, _vp, _vp, _vp, _vp]),
    "bt_device_rcp": (_i32, [_i64, _vp, _vp, _vp]),
    "bt_refine_result": (_i32, [_vp, _f64, _pf64]),
    "bt_plan_set_backward_tol": (_i32, [_vp, _f64]),
    "bt_plan_set_forward_tol": (_i32, [_vp, _f64]),
    "bt_plan_anorm": (_i32, [_vp, _vp]),
    "bt_plan_set_pivot_tol": (_i32, [_vp, _f64]),
    "cyc_plan_create": (_i32, [_pvp, _i64, _i32, _i32, _i32, _i64, _vp]),
    "cyc_factor": (_i32, [_vp, _vp, _vp]),
    "cyc_solve": (_i32, [_vp, _vp, _vp, _i32]),
    "cyc_residual": (_i32, [_vp, _vp, _vp, _vp, _i32]),
    "cyc_refine": (_i32, [_vp, _vp, _vp, _i32, _f64, _i32, ctypes.POINTER(ctypes.c_int),
                          ctypes.POINTER(ctypes.c_double)]),
    "ivp_parareal": (_i32, [_i64, _vp, _vp, _vp, _vp, _vp, _vp, _f64, _i32, _i32, _i32, _i32, _f64, _vp, _vp,
                            ctypes.POINTER(ctypes.c_int), _vp]),
    "ivp_bvm": (_i32, [_i32, _i64, _i64, _f64, _vp, _vp, _vp, _vp, _vp]),
    "pbt_plan_create": (_i32, [_pvp, _i64, _i32, _i32, _i64, _vp]),
    "pbt_factor": (_i32, [_vp, _vp, _vp, _vp]),
    "pbt_solve": (_i32, [_vp, _vp, _vp, _i32]),
    "pbt_residual": (_i32, [_vp, _vp, _vp, _vp, _i32]),
    "pbt_sync": (_i32, [_vp]),
    "pbt_plan_destroy": (None, [_vp]),
    "bt_plan_workspace_size": (_i32, [_i32, _i64, _i32, _i32, _i32, ctypes.POINTER(BtTuning), _pi64]),
    "bt_plan_create_in": (_i32, [_pvp, _i32, _i64, _i32, _i32, _i32, ctypes.POINTER(BtTuning), _vp, _i64, _vp]),
})

_lib = None


def load(path: str = LIB_PATH):
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise ImportError(
            f"{path} is missing: build it with `python -m paper_0912_3678_gb300.build` "
            "(nvcc for sm_103a). There is no CPU fallback.")
    lib = ctypes.CDLL(path)
    for name, (res, args) in SIGNATURES.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


class BtError(RuntimeError):
    def __init__(self, code: int, what: str):
        self.code = code
        self.name = BT_STATUS.get(code, f"status {code}")
        super().__init__(f"{what}: {self.name}")


def check(code: int, what: str) -> int:
    if code != 0:
        raise BtError(code, what)
    return code
