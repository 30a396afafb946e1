"""Symmetric CRS (Sect. 1.3.1): the library's symmetric handle, which stores the
upper triangle with the diagonal once, against the oracle's symmetric loop and
against the plain product of the full matrix.  Irregular upper triangles (empty
rows, rows without a diagonal, repeated entries, unsorted columns) under several
plans of the upper-triangle pass, every alpha/beta form, integer bit-exactness,
the 2D and 3D Laplacians and the Hamiltonian-like matrix at full size, FP32
storage, new values, deterministic results, and the calls a symmetric handle
does not support."""
import ctypes

import numpy as np
import pytest

import oracle
from paper_1106_5908_gb300 import workloads as W
from gpu_util import assert_bitexact, assert_within, dev, host, need_gpu

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

FORMS = [(1.0, 0.0), (-0.75, 1.0), (2.0, -0.5), (0.0, 2.0)]


@pytest.fixture(autouse=True)
def _gpu():
    need_gpu()


def sym(U, dtype=None):
    from paper_1106_5908_gb300 import Matrix
    return Matrix.from_symmetric_upper(U.row_ptr, U.col_idx, U.val, dtype=dtype)


@pytest.mark.parametrize("n", [1, 2, 64, 3000, 20000])
@pytest.mark.parametrize("plan", [None, (4, 7), (0, 15), (5, 4096), (6, 9)])
def test_symmetric_random(n, plan):
    U = W.random_symmetric_upper(n, seed=n + 3, max_len=12)
    M = sym(U)
    if plan is not None:
        M.set_plan(*plan)
    x = W.uniform(n, 5)
    y0 = W.uniform(n, 6)
    for alpha, beta in FORMS:
        ref, bound = oracle.spmv_sym(*U.astuple(), x, alpha, beta, y0, with_bound=True)
        y = dev(y0)
        M.apply(dev(x), y, alpha, beta)
        assert_within(host(y), ref, bound, 1e-13, f"n={n} plan={plan} a={alpha} b={beta}")


def test_symmetric_integer_bitexact():
    U = W.random_symmetric_upper(5000, seed=9, integer=True, max_len=20)
    xi = W.integers(5000, 10).astype(np.float64)
    M = sym(U)
    assert_bitexact(host(M.apply(dev(xi))), oracle.spmv_sym(*U.astuple(), xi), "integer")


@pytest.mark.parametrize("which", ["laplace2d_256", "poisson7_160", "hamiltonian"])
def test_symmetric_full_size(which):
    if which == "laplace2d_256":
        A = W.laplace2d(W.LAPLACE2D_GRID)
    elif which == "poisson7_160":
        A = W.laplace3d(W.POISSON7_GRID)
    else:
        A = W.hamiltonian_like(W.HAMILTONIAN_N, seed=W.SEED_HAMILTONIAN)
    U = W.upper_triangle(A)
    M = sym(U)
    x = W.uniform(A.n_rows, 11)
    ref, bound = oracle.spmv_sym(*U.astuple(), x, with_bound=True)
    y = host(M.apply(dev(x)))
    assert_within(y, ref, bound, 1e-13, f"{which} symmetric vs symmetric oracle")
    full, fbound = oracle.spmv(*A.astuple(), x, with_bound=True)
    assert_within(y, full, fbound, 1e-13, f"{which} symmetric vs full product")
    if which != "hamiltonian":  # integer stencil values: exact
        xi = W.integers(A.n_rows, 12).astype(np.float64)
        assert_bitexact(host(M.apply(dev(xi))), oracle.spmv(*A.astuple(), xi), f"{which} integer")
    y2 = host(M.apply(dev(x)))
    assert np.array_equal(y, y2), "two applies differ"


def test_symmetric_fp32_storage_and_new_values():
    A = W.hamiltonian_like(200000, seed=13)
    U = W.upper_triangle(A)
    M = sym(U, dtype=torch.float32)
    x32 = W.uniform(A.n_rows, 14).astype(np.float32)
    v32 = U.val.astype(np.float32)
    ref, bound = oracle.spmv_sym(U.row_ptr, U.col_idx, v32.astype(np.float64), x32.astype(np.float64),
                                 with_bound=True)
    assert_within(host(M.apply(dev(x32))), ref, bound, 1e-6, "FP32 symmetric")
    v2 = W.uniform(U.nnz, 15).astype(np.float32)
    M.set_values(dev(v2))
    ref2, bound2 = oracle.spmv_sym(U.row_ptr, U.col_idx, v2.astype(np.float64), x32.astype(np.float64),
                                   with_bound=True)
    assert_within(host(M.apply(dev(x32))), ref2, bound2, 1e-6, "FP32 symmetric after new values")
    M64 = sym(U)
    x = W.uniform(A.n_rows, 16)
    M64.apply(dev(x))
    v3 = W.uniform(U.nnz, 17)
    M64.set_values(dev(v3))
    ref3, bound3 = oracle.spmv_sym(U.row_ptr, U.col_idx, v3, x, with_bound=True)
    assert_within(host(M64.apply(dev(x))), ref3, bound3, 1e-13, "FP64 symmetric after new values")


def test_symmetric_unsupported_calls():
    from paper_1106_5908_gb300 import _abi
    U = W.upper_triangle(W.laplace2d(16))
    M = sym(U)
    h = M.handle
    n = U.n_rows
    X = torch.zeros(n, 4, dtype=torch.float64, device="cuda")
    Y = torch.zeros(n, 4, dtype=torch.float64, device="cuda")
    v = torch.zeros(n, dtype=torch.float64, device="cuda")
    p = lambda t: ctypes.c_void_p(t.data_ptr())
    sp = ctypes.c_void_p()
    assert _abi.spmv_split_create(ctypes.byref(sp), h, 4, None, None) == _abi.SPMV_ERR_UNSUPPORTED
    assert _abi.spmm_apply(h, 4, 1.0, p(X), 0.0, p(Y), _abi.SPMV_F64, None) == _abi.SPMV_ERR_UNSUPPORTED
    assert _abi.spmv_backward(h, 1.0, p(v), p(v), p(v), None, None) == _abi.SPMV_ERR_UNSUPPORTED
    arr = (ctypes.c_void_p * 1)(h.value)
    b = ctypes.c_void_p()
    assert _abi.spmv_batched_create(ctypes.byref(b), 1, arr) == _abi.SPMV_ERR_UNSUPPORTED
    st = np.zeros(4)
    assert _abi.spmv_cg(h, p(v), p(v), 1e-10, 10, st.ctypes.data_as(ctypes.c_void_p), None) == _abi.SPMV_ERR_UNSUPPORTED
