"""ctypes binding of the C ABI in ``include/spmv.h``.

Every function of the header is exposed here under the same name with the same
arguments (pointers as Python ints, streams as the integer value of a
``cudaStream_t``); they return the raw ``spmv_status``.  ``check`` turns a status
into an exception.  Nothing here computes: all work runs in ``libspmv.so``.
Loading fails loudly if the library has not been built.
"""
from __future__ import annotations

import ctypes
import os

from .build import LIB_PATH

SPMV_OK = 0
SPMV_ERR_INVALID_ARG = 1
SPMV_ERR_INVALID_INDEX = 2
SPMV_ERR_CUDA = 3
SPMV_ERR_ALLOC = 4
SPMV_ERR_UNSUPPORTED = 5
SPMV_ERR_TIMEOUT = 6
SPMV_ERR_NOT_CONVERGED = 7

SPMV_F64 = 0
SPMV_F32 = 1
SPMV_NOALLOC_MAX_COLS = 1 << 20

# Every entry point declared in include/spmv.h.
EXPORTS = (
    "spmv_status_string", "spmv_version", "spmv_create", "spmv_create_symmetric", "spmv_destroy", "spmv_set_values",
    "spmv_get_info", "spmv_row_histogram", "spmv_set_plan", "spmv_set_accumulator", "spmv_apply", "spmv_split_create",
    "spmv_split_destroy", "spmv_split_get_plan", "spmv_apply_split", "spmv_apply_split_vector",
    "spmv_split_get_halo",
    "spmm_apply", "spmv_backward", "spmv_get_transpose", "spmv_transpose_noalloc", "spmv_batched_create",
    "spmv_batched_destroy", "spmv_batched_apply", "spmv_batched_get_info", "spmv_batched_get_member_plan", "spmv_ir_cg",
    "spmv_cg", "spmv_check_device_error", "spmv_validate_device", "spmv_selftest_wait_timeout",
)


class SpmvError(RuntimeError):
    def __init__(self, status: int, where: str = ""):
        self.status = status
        msg = status_string(status)
        super().__init__(f"{where}: {msg}" if where else msg)


_lib = None

vp = ctypes.c_void_p
i32 = ctypes.c_int32
i64 = ctypes.c_int64
f64 = ctypes.c_double
st = ctypes.c_int


def load() -> ctypes.CDLL:
    """Load ``libspmv.so`` (built by ``build.build()``); raises if it is missing."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(f"{LIB_PATH} is not built: run __graft_entry__.build() "
                           "(nvcc for sm_103a is required; there is no CPU fallback)")
    lib = ctypes.CDLL(LIB_PATH)
    sig = {
        "spmv_status_string": (ctypes.c_char_p, [st]),
        "spmv_version": (i32, []),
        "spmv_create": (st, [vp, i32, i32, i64, vp, vp, vp, st, ctypes.c_int, vp]),
        "spmv_create_symmetric": (st, [vp, i32, i64, vp, vp, vp, st, ctypes.c_int, vp]),
        "spmv_destroy": (None, [vp]),
        "spmv_set_values": (st, [vp, vp, st, vp]),
        "spmv_get_info": (st, [vp, vp, vp, vp, vp]),
        "spmv_row_histogram": (st, [vp, i32, vp]),
        "spmv_set_plan": (st, [vp, i32, i32]),
        "spmv_set_accumulator": (st, [vp, i32]),
        "spmv_apply": (st, [vp, f64, vp, st, f64, vp, st, vp]),
        "spmv_split_create": (st, [vp, vp, i32, vp, vp]),
        "spmv_split_destroy": (None, [vp]),
        "spmv_split_get_plan": (st, [vp, vp, vp, vp, vp, vp, vp, vp]),
        "spmv_apply_split": (st, [vp, f64, vp, f64, vp, vp, vp]),
        "spmv_apply_split_vector": (st, [vp, f64, vp, f64, vp, vp]),
        "spmv_split_get_halo": (st, [vp, vp, vp]),
        "spmm_apply": (st, [vp, i32, f64, vp, f64, vp, st, vp]),
        "spmv_backward": (st, [vp, f64, vp, vp, vp, vp, vp]),
        "spmv_get_transpose": (st, [vp, vp, vp, vp, vp]),
        "spmv_transpose_noalloc": (st, [i32, i32, i64, vp, vp, vp, vp, vp, vp]),
        "spmv_batched_create": (st, [vp, i32, vp]),
        "spmv_batched_get_member_plan": (st, [vp, vp]),
        "spmv_batched_destroy": (None, [vp]),
        "spmv_batched_apply": (st, [vp, f64, vp, f64, vp, vp]),
        "spmv_batched_get_info": (st, [vp, vp]),
        "spmv_ir_cg": (st, [vp, vp, vp, f64, i32, f64, i32, vp, vp]),
        "spmv_cg": (st, [vp, vp, vp, f64, i32, vp, vp]),
        "spmv_check_device_error": (st, [vp, vp]),
        "spmv_validate_device": (st, [i32, i32, i64, vp, vp, vp]),
        "spmv_selftest_wait_timeout": (st, [vp, i64, vp]),
    }
    for name, (res, args) in sig.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


def status_string(status: int) -> str:
    try:
        return load().spmv_status_string(status).decode()
    except Exception:  # library unavailable: describe the code locally
        return f"spmv status {status}"


def check(status: int, where: str = "") -> None:
    if status != SPMV_OK:
        raise SpmvError(status, where)


def _fwd(name):
    def f(*args):
        return getattr(load(), name)(*args)
    f.__name__ = name
    f.__doc__ = f"Direct call of the C entry point {name} (see include/spmv.h)."
    return f


spmv_version = _fwd("spmv_version")
spmv_create = _fwd("spmv_create")
spmv_create_symmetric = _fwd("spmv_create_symmetric")
spmv_destroy = _fwd("spmv_destroy")
spmv_set_values = _fwd("spmv_set_values")
spmv_get_info = _fwd("spmv_get_info")
spmv_row_histogram = _fwd("spmv_row_histogram")
spmv_set_plan = _fwd("spmv_set_plan")
spmv_set_accumulator = _fwd("spmv_set_accumulator")
spmv_apply = _fwd("spmv_apply")
spmv_split_create = _fwd("spmv_split_create")
spmv_split_destroy = _fwd("spmv_split_destroy")
spmv_split_get_plan = _fwd("spmv_split_get_plan")
spmv_apply_split_vector = _fwd("spmv_apply_split_vector")
spmv_apply_split = _fwd("spmv_apply_split")
spmv_split_get_halo = _fwd("spmv_split_get_halo")
spmm_apply = _fwd("spmm_apply")
spmv_backward = _fwd("spmv_backward")
spmv_get_transpose = _fwd("spmv_get_transpose")
spmv_transpose_noalloc = _fwd("spmv_transpose_noalloc")
spmv_batched_create = _fwd("spmv_batched_create")
spmv_batched_get_member_plan = _fwd("spmv_batched_get_member_plan")
spmv_batched_destroy = _fwd("spmv_batched_destroy")
spmv_batched_apply = _fwd("spmv_batched_apply")
spmv_batched_get_info = _fwd("spmv_batched_get_info")
spmv_ir_cg = _fwd("spmv_ir_cg")
spmv_cg = _fwd("spmv_cg")
spmv_check_device_error = _fwd("spmv_check_device_error")
spmv_validate_device = _fwd("spmv_validate_device")
spmv_selftest_wait_timeout = _fwd("spmv_selftest_wait_timeout")
spmv_status_string = _fwd("spmv_status_string")
