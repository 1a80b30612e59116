"""ctypes binding of libtopsolve.so (argument marshalling only).

Every numerical step runs in the CUDA library; this module only converts
arguments.  There is no CPU fallback: if the library is missing or cannot be
loaded, `lib()` raises.
"""
from __future__ import annotations

import ctypes as C
import os

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libtopsolve.so")

TS_OK, TS_PENDING, TS_NOT_CONVERGED = 0, 1, 2
TS_ERR_INVALID, TS_ERR_OOM, TS_ERR_CUDA, TS_ERR_BREAKDOWN = -1, -2, -3, -4
TS_ERR_TIMEOUT, TS_ERR_NOT_SPD, TS_ERR_BUSY = -5, -6, -7
TS_FP64, TS_MIXED_FP32, TS_MIXED_TF32, TS_MIXED_3XTF32 = 0, 1, 2, 3

STATUS_NAMES = {0: "TS_OK", 1: "TS_PENDING", 2: "TS_NOT_CONVERGED", -1: "TS_ERR_INVALID", -2: "TS_ERR_OOM",
                -3: "TS_ERR_CUDA", -4: "TS_ERR_BREAKDOWN", -5: "TS_ERR_TIMEOUT", -6: "TS_ERR_NOT_SPD",
                -7: "TS_ERR_BUSY"}


class TsMesh(C.Structure):
    _fields_ = [("dim", C.c_int), ("nx", C.c_int), ("ny", C.c_int), ("nz", C.c_int), ("blk_x", C.c_int),
                ("blk_y", C.c_int), ("blk_z", C.c_int), ("overlap", C.c_int)]


class TsBcs(C.Structure):
    _fields_ = [("n", C.c_int64), ("dofs", C.POINTER(C.c_int64))]


class TsOptions(C.Structure):
    _fields_ = [("precision", C.c_int), ("tau_scale", C.c_double), ("max_modes", C.c_int), ("rotations", C.c_int),
                ("coarse", C.c_int), ("max_iter", C.c_int), ("warm_start", C.c_int), ("mem_is_device", C.c_int),
                ("energy_tol", C.c_double), ("refine", C.c_int), ("coarse_layout", C.c_int),
                ("coarse_method", C.c_int), ("rand_snapshots", C.c_int), ("rebuild_policy", C.c_int),
                ("rebuild_factor", C.c_double)]


class TsStats(C.Structure):
    _fields_ = [("iters", C.c_int), ("converged", C.c_int), ("rel_res", C.c_double), ("energy_est", C.c_double),
                ("cond_est", C.c_double), ("coarse_dim", C.c_int), ("cap_hits", C.c_int),
                ("eig_unconverged", C.c_int), ("setup_ms", C.c_double), ("solve_ms", C.c_double),
                ("precision", C.c_int), ("first_iters", C.c_int), ("refine_rounds", C.c_int),
                ("precond_age", C.c_int)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


# exported symbols: name -> (restype, argtypes)
SIGNATURES = {
    "ts_options_default": (None, [C.POINTER(TsOptions)]),
    "ts_ctx_create": (C.c_int, [C.c_void_p, C.POINTER(C.c_void_p)]),
    "ts_ctx_destroy": (C.c_int, [C.c_void_p]),
    "ts_last_error": (C.c_char_p, [C.c_void_p]),
    "ts_ctx_kernel_launches": (C.c_int64, [C.c_void_p]),
    "ts_setup": (C.c_int, [C.c_void_p, C.POINTER(TsMesh), C.c_void_p, C.c_double, C.c_double, C.c_double,
                           C.c_double, C.POINTER(TsBcs), C.POINTER(TsOptions), C.POINTER(C.c_void_p)]),
    "ts_solve": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_int, C.c_double, C.POINTER(TsStats)]),
    "ts_apply_K": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p]),
    "ts_apply_M": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p]),
    "ts_apply_K_dot_static": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p]),
    "ts_sensitivity": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.POINTER(C.c_double)]),
    "ts_oc_update": (C.c_int, [C.c_void_p, C.c_void_p, C.c_double, C.c_double, C.c_void_p]),
    "ts_apply_M_parts": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p]),
    "ts_apply_M_block": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_int, C.c_int]),
    "ts_ndof": (C.c_int64, [C.c_void_p]),
    "ts_time_kernel": (C.c_int, [C.c_void_p, C.c_char_p, C.c_int, C.POINTER(C.c_double), C.POINTER(C.c_double),
                                 C.POINTER(C.c_double)]),
    "ts_level1_info": (C.c_int, [C.c_void_p, C.POINTER(C.c_int), C.POINTER(C.c_int64), C.POINTER(C.c_int64)]),
    "ts_coarse_dim": (C.c_int, [C.c_void_p]),
    "ts_coarse_problems": (C.c_int, [C.c_void_p]),
    "ts_coarse_info": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p]),
    "ts_destroy": (C.c_int, [C.c_void_p]),
    "ts_update_density": (C.c_int, [C.c_void_p, C.c_void_p]),
    "ts_ctx_set_slots": (C.c_int, [C.c_void_p, C.c_int]),
    "ts_submit": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_int, C.c_double,
                            C.POINTER(C.c_int64)]),
    "ts_submit_update": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_int,
                                   C.c_double, C.POINTER(C.c_int64)]),
    "ts_poll": (C.c_int, [C.c_void_p, C.c_int64, C.POINTER(TsStats)]),
}

_lib = None


def lib():
    """Loads libtopsolve.so (raises if it was not built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"libtopsolve.so is not built ({LIB_PATH}); run __graft_entry__.build()")
        L = C.CDLL(LIB_PATH)
        for name, (res, args) in SIGNATURES.items():
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _lib = L
    return _lib
