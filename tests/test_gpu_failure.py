"""Failure detection on the GPU without a fault: the device-side CRS check returns
an error status for planted invalid structures (all reads stay in bounds), and the
bounded on-device wait gives up on a barrier that nothing completes, reports
SPMV_ERR_TIMEOUT and leaves the context usable."""
import ctypes
import time

import numpy as np
import pytest

import oracle
from paper_1106_5908_gb300 import workloads as W
from gpu_util import assert_within, dev, host, need_gpu

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(autouse=True)
def _gpu():
    need_gpu()


def validate(rp, col, n_cols):
    from paper_1106_5908_gb300 import _abi
    rpd = torch.as_tensor(np.ascontiguousarray(rp, dtype=np.int32)).cuda()
    cd = torch.as_tensor(np.ascontiguousarray(col, dtype=np.int32)).cuda() if len(col) else None
    nnz = len(col)
    return _abi.spmv_validate_device(len(rp) - 1, n_cols, nnz, ctypes.c_void_p(rpd.data_ptr()),
                                     ctypes.c_void_p(cd.data_ptr()) if cd is not None else None,
                                     ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))


def test_validate_device_accepts_valid_structures():
    from paper_1106_5908_gb300 import _abi
    for A in (W.laplace2d(64, 64), W.hamiltonian_like(20000, seed=2),
              W.random_csr(500, 300, seed=1, max_len=20)):
        assert validate(A.row_ptr, A.col_idx, A.n_cols) == _abi.SPMV_OK
    assert validate(np.zeros(5, np.int32), np.zeros(0, np.int32), 3) == _abi.SPMV_OK  # empty rows


@pytest.mark.parametrize("mistake", ["first_nonzero", "decreasing", "last_not_nnz", "negative_col",
                                     "col_too_large"])
def test_validate_device_rejects_planted_mistakes(mistake):
    from paper_1106_5908_gb300 import _abi
    A = W.hamiltonian_like(20000, seed=3)
    rp, col = A.row_ptr.copy(), A.col_idx.copy()
    if mistake == "first_nonzero":
        rp[0] = 1
    elif mistake == "decreasing":
        rp[777] = rp[778] + 1
    elif mistake == "last_not_nnz":
        rp[-1] -= 1
    elif mistake == "negative_col":
        col[12345] = -1
    else:
        col[-1] = A.n_cols
    assert validate(rp, col, A.n_cols) == _abi.SPMV_ERR_INVALID_INDEX


def test_validate_device_rejects_bad_arguments():
    from paper_1106_5908_gb300 import _abi
    assert _abi.spmv_validate_device(-1, 3, 0, None, None, None) == _abi.SPMV_ERR_INVALID_ARG
    assert _abi.spmv_validate_device(3, 3, 0, None, None, None) == _abi.SPMV_ERR_INVALID_ARG


def test_bounded_wait_times_out_and_context_survives():
    from paper_1106_5908_gb300 import Matrix, _abi
    A = W.laplace2d(128, 128)
    M = Matrix.from_csr(A.row_ptr, A.col_idx, A.val, A.n_cols)
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    for limit_ns in (20_000_000, 1_000_000):
        t0 = time.perf_counter()
        st = _abi.spmv_selftest_wait_timeout(M.handle, limit_ns, stream)
        elapsed = time.perf_counter() - t0
        assert st == _abi.SPMV_ERR_TIMEOUT, _abi.status_string(st)
        assert limit_ns * 1e-9 <= elapsed < 2.0
        assert _abi.spmv_check_device_error(M.handle, stream) == _abi.SPMV_OK  # cleared
    assert _abi.spmv_selftest_wait_timeout(M.handle, 10, stream) == _abi.SPMV_ERR_INVALID_ARG
    assert _abi.spmv_selftest_wait_timeout(M.handle, 2_000_000_000, stream) == _abi.SPMV_ERR_INVALID_ARG
    # the context is usable: a product right after matches the oracle
    x = W.uniform(A.n_cols, 1)
    ref, bound = oracle.spmv(*A.astuple(), x, with_bound=True)
    assert_within(host(M.apply(dev(x))), ref, bound, 1e-13, "after the timeout self-test")
    M.check_device_error()
