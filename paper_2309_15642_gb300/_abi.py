"""ctypes declarations of the C ABI in ``include/gpeps.h`` (argument marshalling only)."""
from __future__ import annotations

import ctypes
import os
from ctypes import POINTER, c_char_p, c_double, c_int, c_int8, c_int32, c_int64, c_size_t, c_void_p

LIB_PATH = os.path.join(os.path.dirname(os.path.abspath(__file__)), "libgpeps.so")

GPEPS_OK, GPEPS_EINVAL, GPEPS_ECUDA, GPEPS_ENOCONV, GPEPS_ENUMERIC, GPEPS_ENOMEM = range(6)
GPEPS_FLAG_NOCONV, GPEPS_FLAG_NUMERIC = 1, 2
GPEPS_C128, GPEPS_MIXED_C64 = 0, 1

# every symbol the header declares, with (restype, argtypes)
SIGNATURES = {
    "gpeps_create": (c_int, [c_void_p, c_int32, c_int32, c_int32, c_void_p, POINTER(c_void_p)]),
    "gpeps_query_workspace": (c_int, [c_void_p, POINTER(c_size_t), POINTER(c_size_t)]),
    "gpeps_bind": (c_int, [c_void_p, c_void_p, c_void_p]),
    "gpeps_reset": (c_int, [c_void_p]),
    "gpeps_kick": (c_int, [c_void_p, c_void_p, c_int32]),
    "gpeps_zz_layer": (c_int, [c_void_p, c_int32]),
    "gpeps_zz_layer_profiled": (c_int, [c_void_p, c_int32, POINTER(ctypes.c_float)]),
    "gpeps_step_profiled": (c_int, [c_void_p, c_void_p, c_int32, POINTER(ctypes.c_float)]),
    "gpeps_set_jacobi": (c_int, [c_void_p, c_double, c_double, c_double, c_double, c_int32, c_int32]),
    "gpeps_set_levels": (c_int, [c_void_p, c_double, c_int32]),
    "gpeps_set_wait_limit": (c_int, [c_void_p, c_int64]),
    "gpeps_inverse_steps": (c_int, [c_void_p, c_int32, c_void_p, c_int32]),
    "gpeps_jacobi_work": (c_int, [c_void_p, POINTER(c_int64)]),
    "gpeps_set_schedule": (c_int, [c_void_p, c_int32]),
    "gpeps_set_tensor_cores": (c_int, [c_void_p, c_int32]),
    "gpeps_n_colours": (c_int, [c_void_p, POINTER(c_int32)]),
    "gpeps_expect_z": (c_int, [c_void_p, c_void_p, c_void_p]),
    "gpeps_step": (c_int, [c_void_p, c_int32, c_void_p, c_int32, c_void_p]),
    "gpeps_status": (c_int, [c_void_p, POINTER(c_int32)]),
    "gpeps_lambda": (c_int, [c_void_p, c_int32, c_int32, POINTER(c_double)]),
    "gpeps_site_layout": (c_int, [c_void_p, c_int32, c_int32, POINTER(c_int64), POINTER(c_int32),
                                  POINTER(c_int32)]),
    "gpeps_lambda_layout": (c_int, [c_void_p, c_int32, c_int32, POINTER(c_int64)]),
    "gpeps_query_grad_workspace": (c_int, [c_void_p, c_int32, c_int32, POINTER(c_size_t)]),
    "gpeps_grad": (c_int, [c_void_p, c_void_p, c_int32, c_int32, c_void_p, c_void_p, c_void_p, c_void_p,
                           c_size_t]),
    "gpeps_query_bp_workspace": (c_int, [c_void_p, c_int32, POINTER(c_size_t)]),
    "gpeps_bp_regauge": (c_int, [c_void_p, c_int32, c_double, c_void_p, c_size_t, POINTER(c_int32),
                                 POINTER(c_double), c_void_p]),
    "gpeps_sizes": (c_int, [c_void_p, POINTER(c_int64), POINTER(c_int64)]),
    "gpeps_sweeps": (c_int, [c_void_p, POINTER(c_int64), POINTER(c_int64), POINTER(c_int64)]),
    "gpeps_bond_phase_cycles": (c_int, [c_void_p, POINTER(c_int64)]),
    "gpeps_selftest_rotation": (c_int, [c_int32, c_int32, c_void_p, c_void_p, c_void_p]),
    "gpeps_bond_update_noalloc": (c_int, [c_int32, c_int32, c_void_p, c_int32, c_int32, c_void_p, c_int32,
                                          c_int32, c_void_p, POINTER(c_double), c_void_p, POINTER(c_int32)]),
    "gpeps_destroy": (c_int, [c_void_p]),
    "gpeps_error_string": (c_char_p, [c_int]),
    "gpeps_last_cuda_error": (c_char_p, []),
}


class GraphC(ctypes.Structure):
    _fields_ = [("n_qubits", c_int32), ("n_edges", c_int32),
                ("edges", POINTER(c_int32)), ("colour", POINTER(c_int8))]


class GpepsError(RuntimeError):
    def __init__(self, status, where, lib=None):
        msg = f"{where}: status {status}"
        if lib is not None:
            msg += " (" + lib.gpeps_error_string(status).decode() + ")"
            if status == GPEPS_ECUDA:
                msg += ": " + lib.gpeps_last_cuda_error().decode()
        super().__init__(msg)
        self.status = status


_LIB = None


def load():
    """Load ``libgpeps.so``; raises if it has not been built (there is no fallback)."""
    global _LIB
    if _LIB is not None:
        return _LIB
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"{LIB_PATH} is missing: run paper_2309_15642_gb300._build.build() "
                          "(the CUDA library is required; there is no CPU path)")
    lib = ctypes.CDLL(LIB_PATH)
    for name, (res, args) in SIGNATURES.items():
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    _LIB = lib
    return lib


def check(status, where):
    if status != GPEPS_OK:
        raise GpepsError(status, where, _LIB)
