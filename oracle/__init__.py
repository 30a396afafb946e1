"""Oracle for the CRS spMVM of Schubert, Fehske, Hager and Wellein (2011).

TEST INFRASTRUCTURE ONLY.  Plain, slow, obviously correct CPU statements of every
operation the GPU library performs, in FP64.  Only ``tests/``, the smoke check and
the CPU-baseline leg of the benchmark may import this package; the library itself
never does, and it shares no code with the CUDA path.

The arithmetic lives in ``spmv_oracle.c`` (compiled with ``-ffp-contract=off`` so
every product and sum is rounded on its own, as the plain definition reads); this
module only marshals numpy arrays.  Each function names the passage it follows.

Parity status: every function here is pinned by ``tests/test_oracle_*.py`` against
dense or brute-force references, closed forms, invariants or the paper's printed
numbers; none is "parity unpinned".
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "spmv_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

_i32p = np.ctypeslib.ndpointer(dtype=np.int32, flags="C_CONTIGUOUS")
_i64p = np.ctypeslib.ndpointer(dtype=np.int64, flags="C_CONTIGUOUS")
_f64p = np.ctypeslib.ndpointer(dtype=np.float64, flags="C_CONTIGUOUS")


def build(force: bool = False) -> str:
    """Compile ``spmv_oracle.c`` into ``liboracle.so`` (plain gcc, OpenMP for the
    timed node-level variant only)."""
    with _lock:
        if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
            tmp = _LIB + f".tmp{os.getpid()}"
            cmd = ["gcc", "-O2", "-ffp-contract=off", "-fno-fast-math", "-fopenmp",
                   "-fPIC", "-shared", "-o", tmp, _SRC, "-lm"]
            subprocess.run(cmd, check=True)
            os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    if _lib is not None:
        return _lib
    build()
    lib = ctypes.CDLL(_LIB)
    i32, i64, f64 = ctypes.c_int32, ctypes.c_int64, ctypes.c_double
    vp = ctypes.c_void_p
    lib.oracle_spmv.argtypes = [i32, _i32p, _i32p, _f64p, _f64p, f64, f64, _f64p, vp]
    lib.oracle_spmv.restype = None
    lib.oracle_spmv_omp.argtypes = [i32, _i32p, _i32p, _f64p, _f64p, f64, f64, _f64p]
    lib.oracle_spmv_omp.restype = None
    lib.oracle_num_threads.argtypes = []
    lib.oracle_num_threads.restype = ctypes.c_int
    lib.oracle_spmm.argtypes = [i32, _i32p, _i32p, _f64p, i32, _f64p, f64, f64, _f64p, vp]
    lib.oracle_spmm.restype = None
    lib.oracle_transpose.argtypes = [i32, i32, _i32p, _i32p, _i32p, _i32p, _i32p]
    lib.oracle_transpose.restype = None
    lib.oracle_backward.argtypes = [i32, i32, _i32p, _i32p, _f64p, f64, _f64p, _f64p, vp, vp, vp]
    lib.oracle_backward.restype = None
    lib.oracle_split_blocks.argtypes = [i32, _i32p, i32, _i32p]
    lib.oracle_split_blocks.restype = None
    lib.oracle_split_halo.argtypes = [i32, i32, _i32p, _i32p, i32, _i32p, _i32p, vp, vp, vp]
    lib.oracle_split_halo.restype = i64
    lib.oracle_cg.argtypes = [i32, _i32p, _i32p, _f64p, _f64p, f64, i32, _f64p]
    lib.oracle_cg.restype = i32
    lib.oracle_row_histogram.argtypes = [i32, _i32p, i32, _i64p]
    lib.oracle_row_histogram.restype = None
    _lib = lib
    return lib


def _ptr(a):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


def _crs(row_ptr, col_idx, val):
    rp = np.ascontiguousarray(row_ptr, dtype=np.int32)
    ci = np.ascontiguousarray(col_idx, dtype=np.int32)
    v = np.ascontiguousarray(val, dtype=np.float64)  # FP32 storage upcasts exactly
    if rp.ndim != 1 or rp.size < 1:
        raise ValueError("row_ptr must have n_rows+1 entries")
    if ci.size < rp[-1] or v.size < rp[-1]:
        raise ValueError("col_idx/val shorter than row_ptr[-1]")
    if ci.size == 0:
        ci = np.zeros(1, np.int32)
    if v.size == 0:
        v = np.zeros(1, np.float64)
    return rp, ci, v


def spmv(row_ptr, col_idx, val, x, alpha=1.0, beta=0.0, y=None, with_bound=False):
    """Listing 1 (Sect. 1.2) generalised to y = alpha*A*x + beta*y.

    Returns y (FP64); with ``with_bound`` also the per-row tolerance scale
    |alpha|*sum_k |val_k x_col(k)| + |beta*y_in|."""
    lib = _load()
    rp, ci, v = _crs(row_ptr, col_idx, val)
    n = rp.size - 1
    xx = np.ascontiguousarray(x, dtype=np.float64)
    if xx.size == 0:
        xx = np.zeros(1, np.float64)
    out = np.zeros(max(n, 1), np.float64)
    if y is not None and beta != 0.0:
        out[:n] = np.asarray(y, dtype=np.float64)
    bound = np.zeros(max(n, 1), np.float64) if with_bound else None
    lib.oracle_spmv(n, rp, ci, v, xx, float(alpha), float(beta), out, _ptr(bound))
    if with_bound:
        return out[:n], bound[:n]
    return out[:n]


def spmv_omp(row_ptr, col_idx, val, x, y_out, alpha=1.0, beta=0.0):
    """Sect. 2 node-level variant (OpenMP over rows), writing into ``y_out``; for the
    timed CPU baseline.  Returns the thread count used."""
    lib = _load()
    lib.oracle_spmv_omp(y_out.size, row_ptr, col_idx, val, x, float(alpha), float(beta), y_out)
    return lib.oracle_num_threads()


def num_threads() -> int:
    return _load().oracle_num_threads()


def spmm(row_ptr, col_idx, val, X, alpha=1.0, beta=0.0, Y=None, with_bound=False):
    """Block vectors: column-by-column application of Listing 1 to X (n_cols x nrhs,
    row-major/interleaved)."""
    lib = _load()
    rp, ci, v = _crs(row_ptr, col_idx, val)
    n = rp.size - 1
    XX = np.ascontiguousarray(X, dtype=np.float64)
    nrhs = XX.shape[1]
    out = np.zeros((max(n, 1), nrhs), np.float64)
    if Y is not None and beta != 0.0:
        out[:n] = np.asarray(Y, dtype=np.float64)
    bound = np.zeros_like(out) if with_bound else None
    if XX.size == 0:
        XX = np.zeros((1, nrhs), np.float64)
    lib.oracle_spmm(n, rp, ci, v, nrhs, XX.reshape(-1), float(alpha), float(beta),
                    out.reshape(-1), _ptr(bound))
    if with_bound:
        return out[:n], bound[:n]
    return out[:n]


def transpose(row_ptr, col_idx, n_cols):
    """Transposed CRS (rows of A^T listed by increasing original position k) and the
    permutation perm[p] = k.  Returns (rowT_ptr, colT_idx, perm)."""
    lib = _load()
    rp = np.ascontiguousarray(row_ptr, dtype=np.int32)
    ci = np.ascontiguousarray(col_idx, dtype=np.int32)
    n = rp.size - 1
    nnz = int(rp[-1])
    rpt = np.zeros(n_cols + 1, np.int32)
    cit = np.zeros(max(nnz, 1), np.int32)
    perm = np.zeros(max(nnz, 1), np.int32)
    if ci.size == 0:
        ci = np.zeros(1, np.int32)
    lib.oracle_transpose(n, int(n_cols), rp, ci, rpt, cit, perm)
    return rpt, cit[:nnz], perm[:nnz]


def backward(row_ptr, col_idx, val, n_cols, g, x, alpha=1.0, with_bound=False):
    """Reverse pass of g^T(alpha*A(val)*x): grad_x = alpha*A^T g (scatter form) and
    grad_val[k] = alpha*g[row k]*x[col k]."""
    lib = _load()
    rp, ci, v = _crs(row_ptr, col_idx, val)
    n = rp.size - 1
    nnz = int(rp[-1])
    gg = np.ascontiguousarray(g, dtype=np.float64)
    xx = np.ascontiguousarray(x, dtype=np.float64)
    if gg.size == 0:
        gg = np.zeros(1)
    if xx.size == 0:
        xx = np.zeros(1)
    gx = np.zeros(max(n_cols, 1), np.float64)
    gv = np.zeros(max(nnz, 1), np.float64)
    bound = np.zeros(max(n_cols, 1), np.float64) if with_bound else None
    lib.oracle_backward(n, int(n_cols), rp, ci, v, float(alpha), gg, xx, _ptr(gx), _ptr(gv), _ptr(bound))
    if with_bound:
        return gx[:n_cols], gv[:nnz], bound[:n_cols]
    return gx[:n_cols], gv[:nnz]


def split_blocks(row_ptr, nblocks):
    """Sect. 3.2 row-block distribution with balanced nonzeros (block starts)."""
    lib = _load()
    rp = np.ascontiguousarray(row_ptr, dtype=np.int32)
    out = np.zeros(nblocks + 1, np.int32)
    lib.oracle_split_blocks(rp.size - 1, rp, int(nblocks), out)
    return out


def split_halo(row_ptr, col_idx, n_cols, block_start):
    """Sect. 3.2 halo bookkeeping: per block, the sorted distinct columns outside the
    block's own range.  Returns (halo_count, halo_map, nnz_local, nnz_nonlocal)."""
    lib = _load()
    rp = np.ascontiguousarray(row_ptr, dtype=np.int32)
    ci = np.ascontiguousarray(col_idx, dtype=np.int32)
    if ci.size == 0:
        ci = np.zeros(1, np.int32)
    bs = np.ascontiguousarray(block_start, dtype=np.int32)
    nb = bs.size - 1
    cnt = np.zeros(nb, np.int32)
    nl = np.zeros(nb, np.int64)
    nn = np.zeros(nb, np.int64)
    total = lib.oracle_split_halo(rp.size - 1, int(n_cols), rp, ci, nb, bs, cnt, None, _ptr(nl), _ptr(nn))
    hmap = np.zeros(max(int(total), 1), np.int32)
    lib.oracle_split_halo(rp.size - 1, int(n_cols), rp, ci, nb, bs, cnt, _ptr(hmap), None, None)
    return cnt, hmap[: int(total)], nl, nn


def cg(row_ptr, col_idx, val, b, tol=1e-12, maxit=10000):
    """Textbook FP64 conjugate gradients (x0 = 0).  Returns (x, iterations)."""
    lib = _load()
    rp, ci, v = _crs(row_ptr, col_idx, val)
    n = rp.size - 1
    bb = np.ascontiguousarray(b, dtype=np.float64)
    x = np.zeros(n, np.float64)
    it = lib.oracle_cg(n, rp, ci, v, bb, float(tol), int(maxit), x)
    return x, int(it)


def row_histogram(row_ptr, nbins):
    """Counts of rows by length (last bin collects the longer rows)."""
    lib = _load()
    rp = np.ascontiguousarray(row_ptr, dtype=np.int32)
    out = np.zeros(nbins, np.int64)
    lib.oracle_row_histogram(rp.size - 1, rp, int(nbins), out)
    return out


def residual(row_ptr, col_idx, val, b, x):
    """r = b - A x with the plain kernel (alpha = -1, beta = 1)."""
    return spmv(row_ptr, col_idx, val, x, alpha=-1.0, beta=1.0, y=b)
