"""ctypes declarations of include/hfmm.h (argument marshalling only)."""
from __future__ import annotations

import ctypes
import os

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libhfmm.so")

IMPEDANCE, TWO_LAYER, THREE_LAYER = 0, 1, 2
FP64, MIXED = 0, 1
PART_NEAR_FREE, PART_FAR_FREE, PART_FAR_REACT, PART_NEAR_REACT, PART_ALL = 1, 2, 4, 8, 15
MAX_LEVELS = 24

STATUS = {0: "HFMM_OK", 1: "HFMM_ERR_INVALID_ARG", 2: "HFMM_ERR_UNSUPPORTED", 3: "HFMM_ERR_OOM",
          4: "HFMM_ERR_CUDA", 5: "HFMM_ERR_NUMERICS", 6: "HFMM_ERR_TIMEOUT"}

# every entry point declared in include/hfmm.h
EXPORTS = ["hfmm_options_default", "hfmm_plan_create", "hfmm_apply", "hfmm_apply_parts",
           "hfmm_apply_adjoint", "hfmm_plan_get_info", "hfmm_plan_get_tree",
           "hfmm_plan_get_pairs", "hfmm_plan_destroy", "hfmm_status_string", "hfmm_last_error",
           "hfmm_debug_bessel", "hfmm_plan_get_stage_times", "hfmm_debug_green_f32",
           "hfmm_leaf_order_noalloc", "hfmm_apply_grad", "hfmm_batch_create", "hfmm_batch_apply",
           "hfmm_batch_get_plan", "hfmm_batch_destroy", "hfmm_debug_wait_timeout", "hfmm_plan_get_leaf_down",
           "hfmm_batch_device_error", "hfmm_batch_apply_grad", "hfmm_solve", "hfmm_plan_get_boxes",
           "hfmm_plan_get_lists"]
NUM_STAGES = 8
STAGES = ["gather", "p2m", "m2m", "down", "l2p", "p2p", "direct", "scatter"]
FLAG_PROFILE = 1
FLAG_SIMT_M2L = 2
FLAG_AUTOTUNE = 4
FLAG_PERSISTENT = 8
FLAG_DENSE_M2L = 16
FLAG_ADAPTIVE = 32


class HfmmError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{STATUS.get(status, status)}: {msg}")
        self.status = status


class hfmm_medium(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int32), ("reserved", ctypes.c_int32), ("k", ctypes.c_double * 3),
                ("d", ctypes.c_double), ("alpha", ctypes.c_double)]


class hfmm_options(ctypes.Structure):
    _fields_ = [("tol", ctypes.c_double), ("p", ctypes.c_int32), ("leaf_size", ctypes.c_int32),
                ("levels", ctypes.c_int32), ("precision", ctypes.c_int32), ("max_rhs", ctypes.c_int32),
                ("flags", ctypes.c_int32), ("spin_limit", ctypes.c_int64), ("quad_scale", ctypes.c_double),
                ("small_rhs", ctypes.c_int32)]


class hfmm_plan_info(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int64), ("levels", ctypes.c_int32), ("lmin", ctypes.c_int32),
                ("p", ctypes.c_int32 * MAX_LEVELS), ("nonempty_leaves", ctypes.c_int64),
                ("v_pairs", ctypes.c_int64), ("r_pairs", ctypes.c_int64),
                ("direct_leaf_pairs", ctypes.c_int64), ("u_pairs", ctypes.c_int64),
                ("x0", ctypes.c_double), ("y0", ctypes.c_double), ("size", ctypes.c_double),
                ("table_bytes", ctypes.c_double), ("buffer_bytes", ctypes.c_double),
                ("plan_ms", ctypes.c_double), ("precision", ctypes.c_int32),
                ("max_rhs", ctypes.c_int32), ("launches_last_apply", ctypes.c_int64),
                ("flops_last_apply", ctypes.c_double * 8), ("bytes_last_apply", ctypes.c_double * 8),
                ("device_error", ctypes.c_int32), ("tensor_levels", ctypes.c_int32),
                ("tune_levels", ctypes.c_int32 * 3), ("tune_ms", ctypes.c_double * 3),
                ("near_tc_blocks", ctypes.c_int64), ("near_simt_leaves", ctypes.c_int64),
                ("leaf_l2p_fused", ctypes.c_int32), ("leaf_tc_width", ctypes.c_int32),
                ("table_check", ctypes.c_double), ("small_rhs", ctypes.c_int32), ("diag_levels", ctypes.c_int32),
                ("diag_check", ctypes.c_double), ("adaptive", ctypes.c_int32), ("tc_run_levels", ctypes.c_int32),
                ("w_pairs", ctypes.c_int64), ("x_pairs", ctypes.c_int64)]


hfmm_plan_t = ctypes.c_void_p
_lib = None


def lib():
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError(f"{LIB_PATH} is not built; run paper_1703_09136_gb300.build.build()")
        L = ctypes.CDLL(LIB_PATH)
        vp, i32, i64, dbl = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_double
        L.hfmm_options_default.argtypes = [vp]
        L.hfmm_options_default.restype = None
        L.hfmm_plan_create.argtypes = [ctypes.POINTER(hfmm_plan_t), i64, vp, vp, vp, vp]
        L.hfmm_apply.argtypes = [hfmm_plan_t, i32, vp, vp, vp]
        L.hfmm_apply_parts.argtypes = [hfmm_plan_t, i32, vp, vp, i32, vp]
        L.hfmm_apply_adjoint.argtypes = [hfmm_plan_t, i32, vp, vp, vp]
        L.hfmm_plan_get_info.argtypes = [hfmm_plan_t, vp]
        L.hfmm_plan_get_tree.argtypes = [hfmm_plan_t, vp, vp, vp]
        L.hfmm_plan_get_pairs.argtypes = [hfmm_plan_t, i32, i32, vp, i64, ctypes.POINTER(i64)]
        L.hfmm_plan_destroy.argtypes = [hfmm_plan_t]
        L.hfmm_status_string.argtypes = [i32]
        L.hfmm_status_string.restype = ctypes.c_char_p
        L.hfmm_last_error.argtypes = []
        L.hfmm_last_error.restype = ctypes.c_char_p
        L.hfmm_debug_bessel.argtypes = [dbl, i32, vp, vp]
        L.hfmm_plan_get_stage_times.argtypes = [hfmm_plan_t, vp]
        L.hfmm_debug_green_f32.argtypes = [i32, vp, vp]
        L.hfmm_leaf_order_noalloc.argtypes = [i64, vp, i32, vp, vp, vp]
        L.hfmm_apply_grad.argtypes = [hfmm_plan_t, i32, vp, vp, vp, vp]
        L.hfmm_batch_create.argtypes = [ctypes.POINTER(vp), i32, vp, vp, vp, vp, vp]
        L.hfmm_batch_apply.argtypes = [vp, i32, vp, vp, i32, vp]
        L.hfmm_batch_get_plan.argtypes = [vp, i32, ctypes.POINTER(hfmm_plan_t)]
        L.hfmm_batch_destroy.argtypes = [vp]
        L.hfmm_debug_wait_timeout.argtypes = [i64, i32]
        L.hfmm_plan_get_leaf_down.argtypes = [hfmm_plan_t, vp, vp]
        L.hfmm_batch_device_error.argtypes = [vp, vp]
        L.hfmm_batch_apply_grad.argtypes = [vp, i32, vp, vp, vp, vp]
        L.hfmm_solve.argtypes = [hfmm_plan_t, vp, vp, vp, dbl, i32, i32, vp, vp, vp]
        L.hfmm_plan_get_boxes.argtypes = [hfmm_plan_t, vp, i64, ctypes.POINTER(i64)]
        L.hfmm_plan_get_lists.argtypes = [hfmm_plan_t, i32, vp, i64, ctypes.POINTER(i64)]
        for name in ("hfmm_plan_create", "hfmm_apply", "hfmm_apply_parts", "hfmm_apply_adjoint",
                     "hfmm_plan_get_info", "hfmm_plan_get_tree", "hfmm_plan_get_pairs",
                     "hfmm_plan_destroy", "hfmm_debug_bessel", "hfmm_plan_get_stage_times",
                     "hfmm_debug_green_f32", "hfmm_leaf_order_noalloc", "hfmm_apply_grad",
                     "hfmm_batch_create", "hfmm_batch_apply", "hfmm_batch_get_plan", "hfmm_batch_destroy",
                     "hfmm_debug_wait_timeout", "hfmm_plan_get_leaf_down", "hfmm_batch_device_error",
                     "hfmm_batch_apply_grad", "hfmm_solve", "hfmm_plan_get_boxes", "hfmm_plan_get_lists"):
            getattr(L, name).restype = i32
        _lib = L
    return _lib


def check(status):
    if status != 0:
        msg = lib().hfmm_last_error().decode(errors="replace")
        raise HfmmError(status, msg)
