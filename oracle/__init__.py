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
numbers; the timed node-level forms (``spmv_omp``, ``spmv_f32``, ``spmv_split``,
``Node``) are pinned bit for bit against the plain loop (or against a literal
Python statement of the split), at every thread count tested; none is "parity
unpinned".
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
_f32p = np.ctypeslib.ndpointer(dtype=np.float32, flags="C_CONTIGUOUS")


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
    lib.oracle_spmv_omp.argtypes = [i32, _i32p, _i32p, _f64p, _f64p, f64, f64, _f64p, i32]
    lib.oracle_spmv_omp.restype = None
    lib.oracle_thread_rows.argtypes = [i32, _i32p, i32, _i32p]
    lib.oracle_thread_rows.restype = None
    lib.oracle_spmv_f32.argtypes = [i32, _i32p, _i32p, _f32p, _f32p, f64, f64, _f32p, i32]
    lib.oracle_spmv_f32.restype = None
    lib.oracle_spmv_split.argtypes = [i32, _i32p, _i32p, _f64p, _f64p, f64, f64, _f64p, i32, _i32p, _i32p,
                                      _i32p, _f64p]
    lib.oracle_spmv_split.restype = None
    lib.oracle_node_create.argtypes = [i32, i32, _i32p, _i32p, _f64p, _f64p, i32, i32, _i32p, _i32p, _i32p]
    lib.oracle_node_create.restype = vp
    lib.oracle_node_destroy.argtypes = [vp]
    lib.oracle_node_destroy.restype = None
    for f in ("oracle_node_spmv", "oracle_node_spmv_f32", "oracle_node_spmv_split"):
        getattr(lib, f).argtypes = [vp, f64, f64]
        getattr(lib, f).restype = None
    lib.oracle_node_set_y.argtypes = [vp, vp, vp]
    lib.oracle_node_set_y.restype = None
    lib.oracle_node_get_y.argtypes = [vp, vp, vp]
    lib.oracle_node_get_y.restype = None
    lib.oracle_node_threads.argtypes = [vp]
    lib.oracle_node_threads.restype = i32
    lib.oracle_num_threads.argtypes = []
    lib.oracle_num_threads.restype = ctypes.c_int
    lib.oracle_spmv_sym.argtypes = [i32, _i32p, _i32p, _f64p, _f64p, f64, f64, _f64p, vp]
    lib.oracle_spmv_sym.restype = None
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


def spmv_sym(row_ptr, col_idx, val, x, alpha=1.0, beta=0.0, y=None, with_bound=False):
    """Symmetric CRS (Sect. 1.3.1): the matrix given by its upper triangle with
    the diagonal; each stored off-diagonal entry serves both of its positions.
    Returns y (FP64); with ``with_bound`` also |alpha|*sum_j |a_ij x_j| + |beta*y|."""
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
    lib.oracle_spmv_sym(n, rp, ci, v, xx, float(alpha), float(beta), out, _ptr(bound))
    if with_bound:
        return out[:n], bound[:n]
    return out[:n]


def thread_rows(row_ptr, nthreads):
    """Sect. 3.5 explicit work distribution: the T+1 bounds of the contiguous,
    nonzero-balanced row chunk of each thread."""
    lib = _load()
    rp = np.ascontiguousarray(row_ptr, dtype=np.int32)
    out = np.zeros(int(nthreads) + 1, np.int32)
    lib.oracle_thread_rows(rp.size - 1, rp, int(nthreads), out)
    return out


def spmv_omp(row_ptr, col_idx, val, x, y_out, alpha=1.0, beta=0.0, nthreads=0):
    """Sect. 2 node-level loop with the Sect. 3.5 work distribution (one contiguous
    nonzero-balanced row chunk per thread), writing into ``y_out`` (FP64, n_rows;
    read when beta != 0).  ``nthreads`` <= 0 uses every available thread.  Returns
    the thread count used."""
    lib = _load()
    rp, ci, v = _crs(row_ptr, col_idx, val)
    xx = np.ascontiguousarray(x, dtype=np.float64)
    if xx.size == 0:
        xx = np.zeros(1, np.float64)
    assert y_out.dtype == np.float64 and y_out.flags["C_CONTIGUOUS"] and y_out.size >= rp.size - 1
    T = int(nthreads) if nthreads and nthreads > 0 else lib.oracle_num_threads()
    yy = y_out if y_out.size > 0 else np.zeros(1, np.float64)
    lib.oracle_spmv_omp(rp.size - 1, rp, ci, v, xx, float(alpha), float(beta), yy, T)
    return T


def spmv_f32(row_ptr, col_idx, val32, x32, alpha=1.0, beta=0.0, y=None, nthreads=1):
    """FP32-stored values and vectors with FP64 accumulation: exact FP64 products
    of the floats, FP64 row sums in increasing k, one rounding of
    alpha*acc + beta*y to float.  Returns y (float32)."""
    lib = _load()
    rp = np.ascontiguousarray(row_ptr, dtype=np.int32)
    ci = np.ascontiguousarray(col_idx, dtype=np.int32)
    v = np.ascontiguousarray(val32, dtype=np.float32)
    xx = np.ascontiguousarray(x32, dtype=np.float32)
    if ci.size == 0:
        ci = np.zeros(1, np.int32)
    if v.size == 0:
        v = np.zeros(1, np.float32)
    if xx.size == 0:
        xx = np.zeros(1, np.float32)
    n = rp.size - 1
    out = np.zeros(max(n, 1), np.float32)
    if y is not None and beta != 0.0:
        out[:n] = np.asarray(y, dtype=np.float32)
    lib.oracle_spmv_f32(n, rp, ci, v, xx, float(alpha), float(beta), out, int(nthreads))
    return out[:n]


def spmv_split(row_ptr, col_idx, val, x, n_cols, block_start, alpha=1.0, beta=0.0, y=None):
    """Sect. 3.4 split form over the row blocks ``block_start`` (Sect. 3.2): halo
    gather, local part (with beta), then the nonlocal part added onto y for rows
    with nonlocal entries.  Returns y (FP64)."""
    lib = _load()
    rp, ci, v = _crs(row_ptr, col_idx, val)
    n = rp.size - 1
    bs = np.ascontiguousarray(block_start, dtype=np.int32)
    cnt, hmap, _, _ = split_halo(rp, ci, n_cols, bs)
    xx = np.ascontiguousarray(x, dtype=np.float64)
    if xx.size == 0:
        xx = np.zeros(1, np.float64)
    out = np.zeros(max(n, 1), np.float64)
    if y is not None and beta != 0.0:
        out[:n] = np.asarray(y, dtype=np.float64)
    hm = np.ascontiguousarray(hmap if hmap.size else np.zeros(1, np.int32), dtype=np.int32)
    halo = np.zeros(max(hmap.size, 1), np.float64)
    lib.oracle_spmv_split(n, rp, ci, v, xx, float(alpha), float(beta), out, bs.size - 1, bs,
                          np.ascontiguousarray(cnt, dtype=np.int32), hm, halo)
    return out[:n]


class Node:
    """The node-level CPU code of Sect. 2 and 3.5 for timing: the matrix, its FP32
    copies and its split form over ``nblocks`` nonzero-balanced row blocks, copied
    into memory first touched by the thread that computes with it, one contiguous
    nonzero-balanced row chunk per thread.  ``spmv``, ``spmv_f32`` and
    ``spmv_split`` run on the node's own vectors (``y``/``y32`` read back with
    ``get_y``)."""

    def __init__(self, row_ptr, col_idx, val, x, n_cols, nthreads=0, nblocks=8):
        lib = _load()
        rp, ci, v = _crs(row_ptr, col_idx, val)
        n = rp.size - 1
        xx = np.ascontiguousarray(x, dtype=np.float64)
        if xx.size == 0:
            xx = np.zeros(1, np.float64)
        nblocks = max(1, int(nblocks))
        bs = split_blocks(rp, nblocks)
        cnt, hmap, _, _ = split_halo(rp, ci, n_cols, bs)
        hm = np.ascontiguousarray(hmap if hmap.size else np.zeros(1, np.int32), dtype=np.int32)
        self.block_start = bs
        self.total_halo = int(cnt.sum())
        self.n_rows = n
        self._lib = lib
        self._h = lib.oracle_node_create(n, int(n_cols), rp, ci, v, xx, int(nthreads), nblocks, bs,
                                         np.ascontiguousarray(cnt, dtype=np.int32), hm)

    @property
    def threads(self) -> int:
        return int(self._lib.oracle_node_threads(self._h))

    def spmv(self, alpha=1.0, beta=0.0):
        self._lib.oracle_node_spmv(self._h, float(alpha), float(beta))

    def spmv_f32(self, alpha=1.0, beta=0.0):
        self._lib.oracle_node_spmv_f32(self._h, float(alpha), float(beta))

    def spmv_split(self, alpha=1.0, beta=0.0):
        self._lib.oracle_node_spmv_split(self._h, float(alpha), float(beta))

    def set_y(self, y=None, y32=None):
        a = None if y is None else np.ascontiguousarray(y, dtype=np.float64)
        b = None if y32 is None else np.ascontiguousarray(y32, dtype=np.float32)
        self._lib.oracle_node_set_y(self._h, _ptr(a), _ptr(b))

    def get_y(self):
        y = np.zeros(max(self.n_rows, 1), np.float64)
        y32 = np.zeros(max(self.n_rows, 1), np.float32)
        self._lib.oracle_node_get_y(self._h, _ptr(y), _ptr(y32))
        return y[: self.n_rows], y32[: self.n_rows]

    def close(self):
        if self._h:
            self._lib.oracle_node_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


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
