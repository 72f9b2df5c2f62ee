"""ctypes loader for libgp.so (the C ABI declared in include/gp.h).

There is no fallback: if the library is missing or cannot be loaded, every call raises.
"""
from __future__ import annotations

import ctypes
import os
import threading

from . import build as _build

GP_OK, GP_ERR_INVALID_ARG, GP_ERR_NOT_PD, GP_ERR_NONFINITE, GP_ERR_OOM, GP_ERR_CUDA, GP_ERR_TIMEOUT, \
    GP_ERR_NO_CONVERGENCE, GP_ERR_NO_DEVICE = range(9)
GP_FP64, GP_FP32, GP_BF16X3, GP_BF16X6, GP_TF32, GP_BF16, GP_FP64_OZAKI = 0, 1, 2, 3, 4, 5, 6
GP_TF32X3 = GP_FP32
# precision names accepted by the Python binding
PRECISIONS = {"fp64": GP_FP64, "fp32": GP_FP32, "tf32x3": GP_TF32X3, "bf16x3": GP_BF16X3, "bf16x6": GP_BF16X6,
              "tf32": GP_TF32, "bf16": GP_BF16, "fp64_ozaki": GP_FP64_OZAKI}

# Every function declared in include/gp.h, with its ctypes signature.
_P, _I32, _I64, _D = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_double


class gp_hyper(ctypes.Structure):
    _fields_ = [("l", ctypes.c_double), ("v", ctypes.c_double), ("s2", ctypes.c_double)]


class gp_config(ctypes.Structure):
    _fields_ = [("tile", ctypes.c_int32), ("precision", ctypes.c_int32), ("ir_tol", ctypes.c_double),
                ("ir_maxit", ctypes.c_int32), ("noisy_prior", ctypes.c_int32), ("timeout_ns", ctypes.c_int64),
                ("grid", ctypes.c_int32), ("withhold_task", ctypes.c_int32), ("withhold_enable", ctypes.c_int32),
                ("tensor_cores", ctypes.c_int32), ("trace", ctypes.c_int32), ("batch_order", ctypes.c_int32),
                ("batch_ctas_per_sm", ctypes.c_int32), ("locality_order", ctypes.c_int32), ("shift", ctypes.c_double),
                ("tile_variant", ctypes.c_int32)]


class gp_batch_desc(ctypes.Structure):
    _fields_ = [("X", ctypes.c_void_p), ("y", ctypes.c_void_p), ("Xs", ctypes.c_void_p), ("n", ctypes.c_int64),
                ("m", ctypes.c_int64), ("D", ctypes.c_int32), ("tile", ctypes.c_int32), ("h", gp_hyper),
                ("mean_out", ctypes.c_void_p), ("cov_out", ctypes.c_void_p)]


class gp_autotune_opts(ctypes.Structure):
    _fields_ = [("tiles", ctypes.c_int32 * 6), ("classes", ctypes.c_int32), ("sample", ctypes.c_int32),
                ("reps", ctypes.c_int32), ("reserved", ctypes.c_int32)]


class gp_autotune_result(ctypes.Structure):
    _fields_ = [("nclass", ctypes.c_int32), ("class_tile", ctypes.c_int32 * 8), ("class_nmax", ctypes.c_int64 * 8),
                ("class_seconds", ctypes.c_double * 8), ("order", ctypes.c_int32), ("ctas_per_sm", ctypes.c_int32),
                ("trials", ctypes.c_int32), ("reserved", ctypes.c_int32), ("seconds_tuned", ctypes.c_double),
                ("seconds_default", ctypes.c_double), ("seconds_spent", ctypes.c_double)]


SIGNATURES = {
    "gp_create": ([ctypes.POINTER(_P), _I32, _P, ctypes.POINTER(gp_config)], _I32),
    "gp_destroy": ([_P], _I32),
    "gp_set_stream": ([_P, _P], _I32),
    "gp_assemble": ([_P, _P, _I64, _I32, gp_hyper, ctypes.POINTER(_P)], _I32),
    "gp_cholesky": ([_P, _P], _I32),
    "gp_predict_mean": ([_P, _P, _P, _P, _I64, _P, ctypes.POINTER(_I32)], _I32),
    "gp_predict_full_cov": ([_P, _P, _P, _I64, _P], _I32),
    "gp_predict_var": ([_P, _P, _P, _I64, _P], _I32),
    "gp_logdet": ([_P, _P, ctypes.POINTER(_D)], _I32),
    "gp_solve": ([_P, _P, _P, _P], _I32),
    "gp_debug_exp_neg": ([_P, _P, _I64, _P], _I32),
    "gp_debug_solve_items": ([_I32, _I32, _I32, _P, _I64], _I64),
    "gp_debug_fx_sqdist": ([_P, _P, _I32, _I32, ctypes.POINTER(_D)], _I32),
    "gp_nlml_grad": ([_P, _P, _P, _I64, _I32, gp_hyper, ctypes.POINTER(_D), ctypes.POINTER(_D)], _I32),
    "gp_batch_create": ([_P, _I32, ctypes.POINTER(gp_batch_desc), ctypes.POINTER(_P)], _I32),
    "gp_batch_run": ([_P, _P], _I32),
    "gp_batch_free": ([_P, _P], _I32),
    "gp_set_batch_schedule": ([_P, _I32, _I32], _I32),
    "gp_factor_stats": ([_P, _P, ctypes.POINTER(ctypes.c_double)], _I32),
    "gp_debug_tile_product": ([_P, _I32, _P, _P, _P, _I32, _I32, _I32, _I32], _I32),
    "gp_batch_predict": ([_P, _I32, ctypes.POINTER(gp_batch_desc), _I32, ctypes.POINTER(ctypes.c_int64)], _I32),
    "gp_batch_autotune": ([_P, _I32, ctypes.POINTER(gp_batch_desc), ctypes.POINTER(gp_autotune_opts),
                           ctypes.POINTER(gp_autotune_result)], _I32),
    "gp_factor_rows": ([_P, _P, _I64, _I64, _P], _I32),
    "gp_alpha": ([_P, _P, _P], _I32),
    "gp_factor_free": ([_P, _P], _I32),
    "gp_sync": ([_P, ctypes.POINTER(_I64)], _I32),
    "gp_status_string": ([_I32], ctypes.c_char_p),
    "gp_launch_count": ([_P], _I64),
    "gp_debug_fail_alloc": ([_I64], None),
    "gp_trace": ([_P, _P, _I64], _I64),
    "gp_predict_mean_noalloc": ([_P, _P, _I64, _I32, gp_hyper, _P, _I64, _P, _P, ctypes.POINTER(_I64)], _I32),
    "gp_schedule_tasks": ([_I32, _I32, _I32, _I32, _I32, _I32, _P, _I64], _I64),
}

_lock = threading.Lock()
_lib = None


def library_path() -> str:
    return _build.LIB


def load(build_if_missing: bool = False) -> ctypes.CDLL:
    """Loads libgp.so (building it first only when asked). Raises if it is not there."""
    global _lib
    with _lock:
        if _lib is None:
            if build_if_missing:
                _build.build()
            if not os.path.exists(_build.LIB):
                raise RuntimeError(f"libgp.so is not built ({_build.LIB}); run __graft_entry__.build()")
            lib = ctypes.CDLL(_build.LIB)
            for name, (args, res) in SIGNATURES.items():
                f = getattr(lib, name)
                f.argtypes = args
                f.restype = res
            _lib = lib
    return _lib
