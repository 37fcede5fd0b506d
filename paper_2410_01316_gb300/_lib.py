"""ctypes loader for libqmcslice.so (the C ABI declared in include/qmcslice.h).

Argument marshalling only: every step of the sum runs in the CUDA library.
There is no CPU fallback; if the library is missing the import of the
binding raises.
"""
from __future__ import annotations

import ctypes
import os
import threading

PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(PKG, "libqmcslice.so")

_lock = threading.Lock()
_lib = None

c_int, c_i64, c_u64, c_dbl, c_vp, c_char_p = (ctypes.c_int, ctypes.c_int64, ctypes.c_uint64, ctypes.c_double,
                                               ctypes.c_void_p, ctypes.c_char_p)

STATUS = {
    0: "QS_OK", 1: "QS_ERR_ARG", 2: "QS_ERR_RANGE", 3: "QS_ERR_NONFINITE", 4: "QS_ERR_OOM",
    5: "QS_ERR_CUDA", 6: "QS_ERR_UNSUPPORTED", 7: "QS_ERR_TIMEOUT",
}
KERNELS = {"gauss": 0, "laplace": 1, "negdist": 2, "matern": 3, "riesz": 4, "tps": 5}
DIRS = {"user": 0, "fibonacci": 1, "orthogonal": 2, "iid": 3, "distance": 4, "sobol": 5}
PROJ = {"auto": 0, "fp32": 1, "fp32_fused": 2, "bf16x3": 3, "tf32": 4}
WINDOWS = {"es": 0, "kb": 1}

# every symbol declared in include/qmcslice.h
EXPORTS = ("qs_plan_create", "qs_plan_destroy", "qs_plan_info", "qs_plan_directions", "qs_sum",
           "qs_sum_host", "qs_check", "qs_status_string", "qs_last_error", "qs_directions", "qs_version",
           "qs_set_timing", "qs_stage_times", "qs_project", "qs_sum_noalloc", "qs_grad",
           "qs_plan_autotune", "qs_plan_set_variant", "qs_batch_create", "qs_batch_destroy", "qs_sum_batched",
           "qs_batch_check", "qs_batch_set_tiling", "qs_plan_variants", "qs_distance_design",
           "qs_distance_energy", "qs_sum_sorted", "qs_grad_sorted", "qs_plan_set_gemm", "qs_plan_gemm",
           "qs_sobol_points", "qs_batch_autotune", "qs_plan_autotune_gemm", "qs_tune_cache_save",
           "qs_tune_cache_load", "qs_tune_cache_clear", "qs_tune_cache_size", "qs_batch_set_mode")


class PlanDesc(ctypes.Structure):
    _fields_ = [
        ("d", c_int), ("kernel", c_int), ("kparam", c_dbl), ("P", c_int), ("dirs", c_int),
        ("seed", c_u64), ("dirs_host", c_vp), ("n_ft", c_int), ("window", c_int),
        ("oversampling", c_dbl), ("radius", c_dbl), ("proj", c_int), ("max_n", c_i64), ("max_m", c_i64),
        ("kparam2", c_dbl), ("window_kind", c_int),
    ]


class Problem(ctypes.Structure):
    _fields_ = [("x", c_vp), ("N", c_i64), ("w", c_vp), ("y", c_vp), ("M", c_i64), ("s", c_vp)]


class QSError(RuntimeError):
    def __init__(self, status: int, where: str, message: str = ""):
        self.status = status
        name = STATUS.get(status, str(status))
        super().__init__(f"{where}: {name}" + (f" ({message})" if message else ""))


def load() -> ctypes.CDLL:
    """Load libqmcslice.so (raises if it has not been built)."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"qmcslice CUDA library not built ({LIB_PATH} missing); "
                               "run paper_2410_01316_gb300.build.build()")
        lib = ctypes.CDLL(LIB_PATH)
        lib.qs_plan_create.argtypes = [ctypes.POINTER(c_vp), ctypes.POINTER(PlanDesc)]
        lib.qs_plan_destroy.argtypes = [c_vp]
        lib.qs_plan_info.argtypes = [c_vp, ctypes.POINTER(c_dbl), ctypes.POINTER(c_int), ctypes.POINTER(c_int),
                                     ctypes.POINTER(c_vp)]
        lib.qs_plan_directions.argtypes = [c_vp, c_vp]
        lib.qs_sum.argtypes = [c_vp, c_vp, c_i64, c_vp, c_vp, c_i64, c_vp, c_vp]
        lib.qs_sum_host.argtypes = [c_vp, c_vp, c_i64, c_vp, c_vp, c_i64, c_vp, c_vp]
        lib.qs_check.argtypes = [c_vp, c_vp]
        lib.qs_status_string.argtypes = [c_int]
        lib.qs_status_string.restype = c_char_p
        lib.qs_last_error.argtypes = []
        lib.qs_last_error.restype = c_char_p
        lib.qs_directions.argtypes = [c_int, c_int, c_int, c_u64, c_vp]
        lib.qs_sobol_points.argtypes = [c_int, c_int, c_u64, c_vp]
        lib.qs_batch_set_mode.argtypes = [c_vp, c_int]
        lib.qs_batch_autotune.argtypes = [c_vp, ctypes.POINTER(Problem), ctypes.POINTER(c_int), c_vp]
        lib.qs_plan_autotune_gemm.argtypes = [c_vp, c_vp, c_i64, ctypes.POINTER(c_int), c_vp]
        lib.qs_tune_cache_save.argtypes = [c_char_p]
        lib.qs_tune_cache_load.argtypes = [c_char_p]
        lib.qs_tune_cache_clear.argtypes = []
        lib.qs_tune_cache_size.argtypes = []
        lib.qs_project.argtypes = [c_vp, c_vp, c_i64, c_vp, c_i64, c_vp]
        lib.qs_batch_create.argtypes = [ctypes.POINTER(c_vp), ctypes.POINTER(c_vp), c_int]
        lib.qs_batch_destroy.argtypes = [c_vp]
        lib.qs_sum_batched.argtypes = [c_vp, ctypes.POINTER(Problem), c_vp]
        lib.qs_batch_check.argtypes = [c_vp, c_vp]
        lib.qs_batch_set_tiling.argtypes = [c_vp, c_int]
        lib.qs_plan_autotune.argtypes = [c_vp, c_vp, c_i64, c_vp, ctypes.POINTER(c_int), c_vp]
        lib.qs_plan_set_variant.argtypes = [c_vp, c_int]
        lib.qs_plan_set_gemm.argtypes = [c_vp, c_int]
        lib.qs_plan_gemm.argtypes = [c_vp, ctypes.POINTER(c_int), ctypes.POINTER(c_int)]
        lib.qs_plan_variants.argtypes = [c_vp, ctypes.POINTER(ctypes.c_uint), ctypes.POINTER(c_int)]
        lib.qs_distance_design.argtypes = [c_vp, c_int, c_int, c_int, c_dbl, ctypes.POINTER(c_dbl), c_vp]
        lib.qs_distance_energy.argtypes = [c_vp, c_int, c_int, ctypes.POINTER(c_dbl), c_vp, c_vp]
        lib.qs_sum_sorted.argtypes = [c_vp, c_vp, c_i64, c_vp, c_vp, c_i64, c_vp, c_vp]
        lib.qs_grad_sorted.argtypes = [c_vp, c_vp, c_i64, c_vp, c_vp, c_i64, c_vp, c_vp, c_vp]
        lib.qs_grad.argtypes = [c_vp, c_vp, c_i64, c_vp, c_vp, c_i64, c_vp, c_vp, c_vp, c_vp, c_vp]
        lib.qs_sum_noalloc.argtypes = [ctypes.POINTER(PlanDesc), c_vp, c_vp, c_i64, c_vp, c_vp, c_i64, c_vp, c_vp]
        lib.qs_set_timing.argtypes = [c_vp, c_int]
        lib.qs_stage_times.argtypes = [c_vp, c_vp, c_int]
        lib.qs_version.argtypes = []
        lib.qs_version.restype = c_char_p
        for name in ("qs_plan_create", "qs_plan_destroy", "qs_plan_info", "qs_plan_directions", "qs_sum",
                     "qs_sum_host", "qs_check", "qs_directions", "qs_set_timing", "qs_stage_times", "qs_project",
                     "qs_sum_noalloc", "qs_grad", "qs_plan_autotune", "qs_plan_set_variant",
                     "qs_batch_create", "qs_batch_destroy", "qs_sum_batched", "qs_batch_check",
                     "qs_batch_set_tiling", "qs_plan_variants", "qs_distance_design", "qs_distance_energy",
                     "qs_sum_sorted", "qs_grad_sorted", "qs_plan_set_gemm", "qs_plan_gemm", "qs_sobol_points",
                     "qs_batch_autotune", "qs_plan_autotune_gemm", "qs_tune_cache_save", "qs_tune_cache_load",
                     "qs_tune_cache_clear", "qs_tune_cache_size", "qs_batch_set_mode"):
            getattr(lib, name).restype = c_int
        _lib = lib
        return lib


def check(status: int, where: str) -> None:
    if status != 0:
        msg = load().qs_last_error().decode(errors="replace")
        raise QSError(status, where, msg)
