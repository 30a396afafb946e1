"""GPU test of spmv_transpose_noalloc, the transposed-CRS build that allocates no
device memory (for callers that cannot call cudaMalloc: latency-bound loops
that must not wait on the allocator, or programs whose device memory is
reserved by another allocator).

Its output is compared bit for bit with the existing entry point
spmv_get_transpose and with the oracle's transposed CRS on calls in a row with
different matrices, so each call after the first runs on the scratch array the
previous one left behind; long columns (one column with an entry in every row)
are among them.  The file name makes pytest collect it last; it passes on its
own in a fresh process as well."""
import ctypes

import numpy as np
import pytest

import oracle
from paper_1106_5908_gb300 import workloads as W
from gpu_util import need_gpu

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def existing_transpose(A):
    from paper_1106_5908_gb300 import Matrix
    M = Matrix.from_csr(A.row_ptr, A.col_idx, A.val, A.n_cols)
    return M.transpose_structure()


def noalloc_transpose(A):
    from paper_1106_5908_gb300 import _abi
    rp = torch.as_tensor(A.row_ptr).cuda()
    ci = torch.as_tensor(A.col_idx).cuda() if A.nnz else torch.zeros(1, dtype=torch.int32, device="cuda")
    rowT = torch.full((A.n_cols + 1,), -7, dtype=torch.int32, device="cuda")
    colT = torch.full((max(A.nnz, 1),), -7, dtype=torch.int32, device="cuda")
    perm = torch.full((max(A.nnz, 1),), -7, dtype=torch.int32, device="cuda")
    st = _abi.spmv_transpose_noalloc(A.n_rows, A.n_cols, A.nnz, ctypes.c_void_p(rp.data_ptr()),
                                     ctypes.c_void_p(ci.data_ptr()), ctypes.c_void_p(rowT.data_ptr()),
                                     ctypes.c_void_p(colT.data_ptr()), ctypes.c_void_p(perm.data_ptr()),
                                     ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert st == _abi.SPMV_OK, _abi.status_string(st)
    torch.cuda.synchronize()
    return rowT.cpu().numpy(), colT.cpu().numpy()[: A.nnz], perm.cpu().numpy()[: A.nnz]


def test_noalloc_transpose_matches_existing_on_two_calls():
    need_gpu()
    first = W.random_csr(3000, 2600, seed=31, max_len=40, long_rows=2, long_len=2000)
    second = W.hamiltonian_like(20000, seed=32)
    third = W.column_heavy_csr(100000, 60000, seed=33, dense=1, medium=20, medium_len=3000)
    for A in (first, second, third, first):
        ref = existing_transpose(A)
        orc = oracle.transpose(A.row_ptr, A.col_idx, A.n_cols)
        got = noalloc_transpose(A)
        for name, g, r, o in zip(("rowT_ptr", "colT_idx", "perm"), got, ref, orc):
            assert g.shape == r.shape == o.shape, name
            assert np.array_equal(g, r), name
            assert np.array_equal(g, o), name


def test_noalloc_transpose_rejects_too_many_columns():
    need_gpu()
    from paper_1106_5908_gb300 import _abi
    n_cols = _abi.SPMV_NOALLOC_MAX_COLS + 1
    rp = torch.zeros(2, dtype=torch.int32, device="cuda")
    rowT = torch.zeros(n_cols + 1, dtype=torch.int32, device="cuda")
    st = _abi.spmv_transpose_noalloc(1, n_cols, 0, ctypes.c_void_p(rp.data_ptr()), None,
                                     ctypes.c_void_p(rowT.data_ptr()), None, None, None)
    assert st == _abi.SPMV_ERR_UNSUPPORTED
    assert int(rowT.abs().sum().item()) == 0  # nothing was written
