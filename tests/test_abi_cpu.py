"""CPU checks of the C ABI: the library builds for sm_103a, loads without a GPU,
exports every entry point include/spmv.h declares, and rejects invalid CRS input
on the host before touching the device."""
import ctypes
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_1106_5908_gb300 import build, _abi
    build.build()
    return _abi.load()


def header_functions():
    src = open(os.path.join(ROOT, "include", "spmv.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b((?:spmv|spmm)_[a-z0-9_]+)\s*\(", src)))


def test_exports_every_declared_symbol(lib):
    names = header_functions()
    assert len(names) >= 20
    for n in names:
        assert hasattr(lib, n), n
    from paper_1106_5908_gb300 import _abi
    assert sorted(_abi.EXPORTS) == names


def test_status_strings(lib):
    for code in range(8):
        s = lib.spmv_status_string(code).decode()
        assert s.startswith("SPMV_")
    assert lib.spmv_version() >= 100


def _create(lib, n_rows, n_cols, rp, ci, val):
    from paper_1106_5908_gb300 import _abi
    h = ctypes.c_void_p()
    rp = np.ascontiguousarray(rp, np.int32)
    ci = np.ascontiguousarray(ci, np.int32)
    val = np.ascontiguousarray(val, np.float64)
    st = lib.spmv_create(ctypes.byref(h), n_rows, n_cols, int(ci.size),
                         rp.ctypes.data_as(ctypes.c_void_p), ci.ctypes.data_as(ctypes.c_void_p),
                         val.ctypes.data_as(ctypes.c_void_p), _abi.SPMV_F64, 0, None)
    return st, h


def test_invalid_crs_rejected_on_host(lib):
    from paper_1106_5908_gb300 import _abi
    ok_rp = [0, 2, 3]
    # row_ptr[0] != 0
    assert _create(lib, 2, 3, [1, 2, 3], [0, 1, 2], [1, 1, 1])[0] == _abi.SPMV_ERR_INVALID_INDEX
    # decreasing row_ptr
    assert _create(lib, 2, 3, [0, 3, 2], [0, 1, 2], [1, 1, 1])[0] == _abi.SPMV_ERR_INVALID_INDEX
    # row_ptr[n] != nnz
    assert _create(lib, 2, 3, [0, 1, 2], [0, 1, 2], [1, 1, 1])[0] == _abi.SPMV_ERR_INVALID_INDEX
    # column out of range (both ends)
    assert _create(lib, 2, 3, ok_rp, [0, 3, 1], [1, 1, 1])[0] == _abi.SPMV_ERR_INVALID_INDEX
    assert _create(lib, 2, 3, ok_rp, [0, -1, 1], [1, 1, 1])[0] == _abi.SPMV_ERR_INVALID_INDEX
    # bad sizes and null pointers
    h = ctypes.c_void_p()
    assert lib.spmv_create(None, 2, 3, 3, None, None, None, 0, 0, None) == _abi.SPMV_ERR_INVALID_ARG
    assert lib.spmv_create(ctypes.byref(h), -1, 3, 0, None, None, None, 0, 0, None) == _abi.SPMV_ERR_INVALID_ARG
    assert lib.spmv_create(ctypes.byref(h), 2, 3, 3, None, None, None, 0, 0, None) == _abi.SPMV_ERR_INVALID_ARG
    assert lib.spmv_create(ctypes.byref(h), 2, 3, 1 << 31, None, None, None, 0, 0, None) == _abi.SPMV_ERR_INVALID_ARG
    assert lib.spmv_create(ctypes.byref(h), 2, 3, 0, None, None, None, 7, 0, None) == _abi.SPMV_ERR_INVALID_ARG


def test_null_handles_rejected(lib):
    from paper_1106_5908_gb300 import _abi
    assert lib.spmv_apply(None, 1.0, None, 0, 0.0, None, 0, None) == _abi.SPMV_ERR_INVALID_ARG
    assert lib.spmm_apply(None, 4, 1.0, None, 0.0, None, 0, None) == _abi.SPMV_ERR_INVALID_ARG
    assert lib.spmv_backward(None, 1.0, None, None, None, None, None) == _abi.SPMV_ERR_INVALID_ARG
    assert lib.spmv_set_plan(None, 0, 15) == _abi.SPMV_ERR_INVALID_ARG
    assert lib.spmv_set_accumulator(None, 0) == _abi.SPMV_ERR_INVALID_ARG
    assert lib.spmv_split_create(None, None, 8, None, None) == _abi.SPMV_ERR_INVALID_ARG
    assert lib.spmv_batched_create(None, 0, None) == _abi.SPMV_ERR_INVALID_ARG
    assert lib.spmv_ir_cg(None, None, None, 1e-12, 50, 1e-4, 200, None, None) == _abi.SPMV_ERR_INVALID_ARG
    lib.spmv_destroy(None)
    lib.spmv_split_destroy(None)
    lib.spmv_batched_destroy(None)


def test_tiler_and_tuner_are_host_logic():
    """The binding refuses to run without the library, and there is no CPU path."""
    import paper_1106_5908_gb300.torch_api as api
    assert not hasattr(api, "cpu_apply")


def test_symmetric_create_rejects_lower_entries_on_host(lib):
    """spmv_create_symmetric takes the upper triangle: an entry left of the
    diagonal, or any CRS mistake, is rejected before the device is touched."""
    from paper_1106_5908_gb300 import _abi

    def create(n, rp, ci):
        h = ctypes.c_void_p()
        rp = np.ascontiguousarray(rp, np.int32)
        ci = np.ascontiguousarray(ci, np.int32)
        val = np.ones(max(ci.size, 1))
        return lib.spmv_create_symmetric(ctypes.byref(h), n, int(ci.size), rp.ctypes.data_as(ctypes.c_void_p),
                                         ci.ctypes.data_as(ctypes.c_void_p), val.ctypes.data_as(ctypes.c_void_p),
                                         _abi.SPMV_F64, 0, None)
    assert create(3, [0, 2, 3, 4], [0, 2, 0, 2]) == _abi.SPMV_ERR_INVALID_INDEX   # (1, 0) lies below
    assert create(3, [0, 2, 3, 4], [0, 3, 1, 2]) == _abi.SPMV_ERR_INVALID_INDEX   # column out of range
    assert create(3, [1, 2, 3, 4], [0, 2, 1, 2]) == _abi.SPMV_ERR_INVALID_INDEX   # row_ptr[0] != 0
    assert lib.spmv_create_symmetric(None, 3, 0, None, None, None, 0, 0, None) == _abi.SPMV_ERR_INVALID_ARG
    assert lib.spmv_create_symmetric(ctypes.byref(ctypes.c_void_p()), -1, 0, None, None, None, 0, 0,
                                     None) == _abi.SPMV_ERR_INVALID_ARG
