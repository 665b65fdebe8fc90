"""ctypes declarations of libmspv.so (the C ABI in include/mspv.h).

Loading fails loudly when the library has not been built: there is no fallback.
"""
from __future__ import annotations

import ctypes
import os

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "lib", "libmspv.so")

OK, EINVAL, ENOMEM, ETOOBIG, EFORMAT, ECUDA, ENOTCONV, EBREAKDOWN = range(8)
STATUS_NAMES = ["MSPV_OK", "MSPV_EINVAL", "MSPV_ENOMEM", "MSPV_ETOOBIG", "MSPV_EFORMAT",
                "MSPV_ECUDA", "MSPV_ENOTCONV", "MSPV_EBREAKDOWN"]
FORMATS = {"coo": 0, "csr": 1, "dia": 2}
VALUE_TYPES = {"f64": 0, "f32": 1, "bf16": 2}


class MatrixInfo(ctypes.Structure):
    _fields_ = [("format", ctypes.c_int32), ("value_type", ctypes.c_int32),
                ("nrows", ctypes.c_int32), ("ncols", ctypes.c_int32), ("nnz", ctypes.c_int64),
                ("ndiags", ctypes.c_int32), ("npad", ctypes.c_int32),
                ("csr_vector", ctypes.c_int32), ("row_max", ctypes.c_int32),
                ("row_mean", ctypes.c_double), ("row_std", ctypes.c_double),
                ("empty_rows", ctypes.c_int64), ("device_bytes", ctypes.c_int64)]


class MspvError(RuntimeError):
    def __init__(self, status: int, message: str):
        self.status = status
        name = STATUS_NAMES[status] if 0 <= status < len(STATUS_NAMES) else str(status)
        super().__init__(f"{name}: {message}")


_lib = None

i32, i64, dbl, vp = ctypes.c_int32, ctypes.c_int64, ctypes.c_double, ctypes.c_void_p
P_I32 = ctypes.POINTER(ctypes.c_int32)
P_DBL = ctypes.POINTER(ctypes.c_double)

SIGNATURES = {
    "mspv_create_coo": (i32, [i32, i32, i64, vp, vp, vp, ctypes.c_int, vp, ctypes.POINTER(vp)]),
    "mspv_convert": (i32, [vp, ctypes.c_int, ctypes.c_int, vp, ctypes.POINTER(vp)]),
    "mspv_spmv": (i32, [vp, vp, vp, vp]),
    "mspv_cg_solve": (i32, [vp, vp, vp, dbl, i32, vp, P_I32, P_DBL]),
    "mspv_cg_solve_ir": (i32, [vp, vp, vp, vp, dbl, dbl, i32, i32, i32, vp, P_I32, P_I32, P_DBL]),
    "mspv_spmv_coo_noalloc": (i32, [i32, i32, i64, vp, vp, vp, vp, vp, vp]),
    "mspv_info": (i32, [vp, ctypes.POINTER(MatrixInfo)]),
    "mspv_export": (i32, [vp, vp, vp, vp, vp]),
    "mspv_destroy": (None, [vp]),
    "mspv_last_error": (ctypes.c_char_p, []),
    "mspv_status_string": (ctypes.c_char_p, [ctypes.c_int]),
    "mspv_csr_vector_width": (i32, [dbl, dbl, i32]),
    "mspv_version": (i32, []),
    "mspv_spmv_add": (i32, [vp, vp, vp, vp]),
    "mspv_spmv_f32": (i32, [vp, vp, vp, vp]),
    "mspv_split_columns": (i32, [vp, i32, vp, ctypes.POINTER(vp), ctypes.POINTER(vp)]),
    "mspv_features": (i32, [vp, vp, vp]),
    "mspv_tune_format": (i32, [vp, i32, vp, vp, ctypes.POINTER(ctypes.c_int)]),
    "mspv_selector_train": (i32, [vp, vp, i32, i32, ctypes.c_float, ctypes.c_uint64, vp, vp]),
    "mspv_selector_predict": (i32, [vp, vp, i32, vp, vp]),
    "mspv_select_format": (i32, [vp, vp, vp, ctypes.POINTER(ctypes.c_int)]),
    "mspv_fp64_fma_rate": (i32, [i64, i32, vp, ctypes.POINTER(dbl)]),
}

NUM_FEATURES = 10
SELECTOR_PARAMS = 5099


def load(path: str = LIB_PATH) -> ctypes.CDLL:
    """Load libmspv.so (once). Raises if it has not been built."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError(f"libmspv.so is not built ({path} missing): run "
                           "`python -c 'import __graft_entry__ as g; g.build()'` first")
    lib = ctypes.CDLL(path)
    for name, (res, args) in SIGNATURES.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


def check(status: int, allow=()):
    if status != OK and status not in allow:
        msg = load().mspv_last_error().decode(errors="replace")
        raise MspvError(status, msg)
    return status
