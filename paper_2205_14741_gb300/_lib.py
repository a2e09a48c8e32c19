"""ctypes declarations of the C ABI in include/smx.h (argument marshalling only).

The shared library is built in-tree (``lib/libsmx.so``) by
``paper_2205_14741_gb300.build``.  There is no fallback: if the library is
missing or fails to load, every call raises.
"""

from __future__ import annotations

import ctypes as C
import os

LIB_PATH = os.path.join(os.path.dirname(os.path.abspath(__file__)), "lib", "libsmx.so")

# smx_status
OK, ERR_ARG, ERR_PATTERN, ERR_NONFINITE, ERR_CUDA, ERR_OOM, ERR_NOCONV, ERR_NOBRACKET, ERR_TIMEOUT, ERR_STATE, \
    ERR_UNSUPPORTED = range(11)
# smx_precision
FP64, FP16X3, FP16, BF16 = range(4)
PRECISIONS = {"fp64": FP64, "fp16x3": FP16X3, "fp16": FP16, "bf16": BF16}
# smx_function: matrix function of a build
FN_DENSITY, FN_INV_SQRT, FN_SQRT, FN_INV, FN_FERMI = 0, 1, 2, 3, 4
FUNCTIONS = {"density": FN_DENSITY, "inv_sqrt": FN_INV_SQRT, "sqrt": FN_SQRT, "inv": FN_INV, "fermi": FN_FERMI}
# learned spectral bound
BOUND_MODEL_FEATURES = 9
BOUND_MODEL_PARAMS = 4930


class Stats(C.Structure):
    _fields_ = [
        ("n_block_cols", C.c_int32),
        ("n", C.c_int64),
        ("nnzb_input", C.c_int64),
        ("nnzb_filtered", C.c_int64),
        ("dim_min", C.c_int32),
        ("dim_max", C.c_int32),
        ("dim_mean", C.c_double),
        ("iters_min", C.c_int32),
        ("iters_max", C.c_int32),
        ("iters_mean", C.c_double),
        ("n_noconv", C.c_int32),
        ("n_bound_fallback", C.c_int32),
        ("bisection_steps", C.c_int32),
        ("flops_ns", C.c_double),
        ("ms_last_build", C.c_double),
        ("mu", C.c_double),
        ("precision", C.c_int32),
        ("fp64_final_iters", C.c_int32),
        ("kernel_launches", C.c_int64),
        ("ns_launches", C.c_int64),
        ("ns_ms_total", C.c_double),
        ("ns_work_n3", C.c_double),
    ]

    def as_dict(self):
        return {name: getattr(self, name) for name, _ in self._fields_}


# name -> (restype, argtypes), in the order of include/smx.h
SIGNATURES = {
    "smx_status_string": (C.c_char_p, [C.c_int]),
    "smx_create": (C.c_int, [C.POINTER(C.c_void_p), C.c_int32, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p,
                             C.c_void_p]),
    "smx_set_values": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int32]),
    "smx_set_filter_threshold": (C.c_int, [C.c_void_p, C.c_double]),
    "smx_set_staging_limit": (C.c_int, [C.c_void_p, C.c_uint64]),
    "smx_set_column_range": (C.c_int, [C.c_void_p, C.c_int32, C.c_int32]),
    "smx_get_gershgorin_interval": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p]),
    "smx_set_mu": (C.c_int, [C.c_void_p, C.c_double]),
    "smx_set_electron_count": (C.c_int, [C.c_void_p, C.c_double, C.c_int32, C.c_double]),
    "smx_set_precision": (C.c_int, [C.c_void_p, C.c_int, C.c_int32]),
    "smx_set_function": (C.c_int, [C.c_void_p, C.c_int]),
    "smx_set_fermi_beta": (C.c_int, [C.c_void_p, C.c_double]),
    "smx_set_symmetrize": (C.c_int, [C.c_void_p, C.c_int32]),
    "smx_set_overlap": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int]),
    "smx_build_density": (C.c_int, [C.c_void_p]),
    "smx_solve_mu": (C.c_int, [C.c_void_p]),
    "smx_get_trace": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p]),
    "smx_get_density": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int32]),
    "smx_get_pattern": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p]),
    "smx_get_stats": (C.c_int, [C.c_void_p, C.POINTER(Stats)]),
    "smx_bound_model_init": (C.c_int, [C.c_void_p, C.c_uint64]),
    "smx_bound_model_set_params": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int32]),
    "smx_bound_model_get_params": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int32]),
    "smx_bound_model_collect": (C.c_int, [C.c_void_p, C.c_int32]),
    "smx_bound_model_train": (C.c_int, [C.c_void_p, C.c_int32, C.c_int32, C.c_float, C.c_void_p]),
    "smx_bound_model_fit": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_int32, C.c_int32, C.c_float,
                                      C.c_void_p, C.c_void_p]),
    "smx_bound_model_predict": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_int32]),
    "smx_set_bound_model": (C.c_int, [C.c_void_p, C.c_int32, C.c_char_p]),
    "smx_bound_model_save": (C.c_int, [C.c_void_p, C.c_char_p]),
    "smx_solve_mu_device": (C.c_int, [C.c_void_p]),
    "smx_selftest_wait_timeout": (C.c_int, [C.c_void_p, C.c_uint32]),
    "smx_reset_counters": (C.c_int, [C.c_void_p]),
    "smx_get_submatrix_info": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p]),
    "smx_dense_density_noalloc": (C.c_int, [C.c_void_p, C.c_int32, C.c_double, C.c_void_p, C.c_void_p]),
    "smx_destroy": (None, [C.c_void_p]),
}

_lib = None


def load() -> C.CDLL:
    """Loads ``libsmx.so`` once and declares every exported function."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(f"{LIB_PATH} is missing: build it with `python -m paper_2205_14741_gb300.build`")
    lib = C.CDLL(LIB_PATH)
    for name, (res, args) in SIGNATURES.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


class SmxError(RuntimeError):
    def __init__(self, status: int, where: str):
        self.status = status
        msg = load().smx_status_string(status).decode()
        super().__init__(f"{where}: {msg} (status {status})")


def check(status: int, where: str) -> None:
    if status != OK:
        raise SmxError(status, where)
