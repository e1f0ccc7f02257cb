"""ctypes declarations of the C ABI in include/amg_b300.h (argument
marshalling only).  Loading fails loudly when libamgb300.so is missing: there
is no CPU fallback."""
from __future__ import annotations

import ctypes as C
import os
import threading

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libamgb300.so")

AMG_OK, AMG_MAXIT, AMG_BREAKDOWN, AMG_NOT_SPD, AMG_NAN = 0, 1, 2, 3, 4
AMG_ERR_ARG, AMG_ERR_BAD_CSR, AMG_ERR_ZERO_DIAG, AMG_ERR_CUDA = -1, -2, -3, -4
AMG_ERR_STALL, AMG_ERR_OOM, AMG_ERR_UNSUPPORTED = -5, -6, -7
AMG_MAX_LEVELS = 32
AMG_DENSE_MAX = 256
AMG_NOALLOC_MAX_N = 1 << 18
AMG_BATCH_MAX_RHS = 8
AMG_TEST_WITHHOLD_COPY, AMG_TEST_WITHHOLD_BARRIER = 1, 2

SOLVERS = {"PCG": 0, "BICGSTAB": 1, "CG": 2, "BICGSTAB_NOPREC": 3}
SMOOTHERS = {"JACOBI": 0, "L1_JACOBI": 1}
PRECISIONS = {"FP64": 0, "MIXED": 1}
LAYOUTS = {"AUTO": 0, "CSR": 1, "WINDOWED": 2, "SLICED_ELL": 3, "ELL_DIRECT": 4, "TILES": 5}
AMG_TYPES = {"AGGREGATION": 0, "CLASSICAL": 1}

# Every symbol the header declares.
EXPORTS = ("amg_config_default", "amg_setup", "amg_resetup", "amg_solve", "amg_adjoint", "amg_vcycle", "amg_get_info",
           "amg_get_level", "amg_get_aggregates", "amg_get_plan", "amg_profile", "amg_profile_summary", "amg_profile_record", "amg_profile_product",
           "amg_setup_batched", "amg_solve_batched", "amg_batch_level", "amg_cg_solve_noalloc", "amg_test_arm_wait_timeout", "amg_narrow_f64", "amg_widen_f32", "amg_free", "amg_status_string", "amg_last_error")


class AmgConfig(C.Structure):
    _fields_ = [("solver", C.c_int), ("smoother", C.c_int), ("omega", C.c_double), ("theta", C.c_double),
                ("coarse_max", C.c_int), ("max_levels", C.c_int), ("rtol", C.c_double), ("max_iter", C.c_int),
                ("max_restarts", C.c_int), ("precision", C.c_int), ("symmetric", C.c_int), ("layout", C.c_int),
                ("adjoint_reuse", C.c_int), ("amg_type", C.c_int), ("fuse_coarse", C.c_int),
                ("device_loop", C.c_int), ("outer_product", C.c_int)]


class AmgInfo(C.Structure):
    _fields_ = [("status", C.c_int), ("iters", C.c_int), ("restarts", C.c_int), ("nlevels", C.c_int),
                ("rel_res_true", C.c_double), ("rel_res_rec", C.c_double),
                ("rows", C.c_int * AMG_MAX_LEVELS), ("nnz", C.c_longlong * AMG_MAX_LEVELS),
                ("operator_complexity", C.c_double), ("setup_ms", C.c_double), ("solve_ms", C.c_double)]


_lock = threading.Lock()
_lib = None


def load() -> C.CDLL:
    """Loads libamgb300.so from the package directory (build it with
    ``python -m paper_2606_09001_b300.build``)."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is missing: build the CUDA library with "
                               "`python -m paper_2606_09001_b300.build` (there is no CPU fallback)")
        L = C.CDLL(LIB_PATH)
        vp, i, ll, d = C.c_void_p, C.c_int, C.c_longlong, C.c_double
        L.amg_config_default.argtypes = [C.POINTER(AmgConfig)]
        L.amg_setup.argtypes = [C.POINTER(AmgConfig), i, ll, vp, vp, vp, vp, C.POINTER(vp)]
        L.amg_resetup.argtypes = [vp, vp, vp]
        L.amg_solve.argtypes = [vp, vp, vp, vp, C.POINTER(AmgInfo)]
        L.amg_adjoint.argtypes = [vp, vp, vp, vp, vp, vp, C.POINTER(AmgInfo)]
        L.amg_vcycle.argtypes = [vp, vp, vp, vp]
        L.amg_get_info.argtypes = [vp, C.POINTER(AmgInfo)]
        L.amg_get_level.argtypes = [vp, i, i, C.POINTER(ll), vp, vp, vp]
        L.amg_get_aggregates.argtypes = [vp, i, vp]
        L.amg_get_plan.argtypes = [vp, i, i, vp]
        L.amg_narrow_f64.argtypes = [vp, vp, C.c_longlong, vp]
        L.amg_widen_f32.argtypes = [vp, vp, C.c_longlong, vp]
        L.amg_profile.argtypes = [vp, i]
        L.amg_profile_summary.argtypes = [vp, C.POINTER(ll), C.POINTER(i)]
        L.amg_profile_record.argtypes = [vp, i, C.c_char_p, i, C.POINTER(i), C.POINTER(ll), C.POINTER(C.c_double),
                                         C.POINTER(C.c_double)]
        L.amg_setup_batched.argtypes = [C.POINTER(AmgConfig), i, vp, i, ll, vp, vp, vp, vp, C.POINTER(vp)]
        L.amg_solve_batched.argtypes = [vp, i, vp, vp, vp, vp, vp, C.POINTER(AmgInfo)]
        L.amg_batch_level.argtypes = [vp, i, C.POINTER(i), vp, vp, vp]
        L.amg_cg_solve_noalloc.argtypes = [i, ll, vp, vp, vp, vp, vp, C.c_double, i, vp, C.POINTER(AmgInfo)]
        L.amg_test_arm_wait_timeout.argtypes = [vp, i]
        L.amg_profile_product.argtypes = [vp, i, C.POINTER(d)]
        L.amg_free.argtypes = [vp]
        L.amg_status_string.argtypes = [i]
        L.amg_status_string.restype = C.c_char_p
        L.amg_last_error.argtypes = []
        L.amg_last_error.restype = C.c_char_p
        for name in EXPORTS:
            if name not in ("amg_status_string", "amg_last_error"):
                getattr(L, name).restype = C.c_int
        _lib = L
        return L


def status_string(code: int) -> str:
    return load().amg_status_string(code).decode()


def last_error() -> str:
    return load().amg_last_error().decode()
