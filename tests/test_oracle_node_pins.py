"""Pins of the oracle's timed node-level forms (Sect. 2 OpenMP outer loop with the
Sect. 3.5 explicit work distribution and first-touch placement), its FP32-storage
form and its split form (Sect. 3.4), against things other than themselves:
the plain single-thread loop bit for bit at every thread count (the row sums are
the same sequence of operations whatever the chunking), a literal Python
statement of the split on tiny inputs, exact integer arithmetic, and the
nonzero-balanced chunk rule written with ``np.searchsorted``.  CPU only."""
import numpy as np
import pytest

import oracle
from paper_1106_5908_gb300 import workloads as W

ALPHA_BETA = [(1.0, 0.0), (-0.5, 1.0), (2.0, -3.0), (0.0, 1.5), (1.0, 1.0)]
THREADS = [1, 2, 3, 5, 0]  # 0: every available thread
SHAPES = [(0, 0), (1, 1), (5, 1), (17, 33), (64, 64), (200, 150), (301, 301)]


def irregular(shape, seed):
    return W.random_csr(*shape, seed=seed, empty_frac=0.3, dup_frac=0.2)


@pytest.mark.parametrize("nt", [1, 2, 3, 4, 7, 16])
@pytest.mark.parametrize("seed", [1, 2])
def test_thread_rows_is_the_nonzero_balanced_rule(nt, seed):
    A = W.random_csr(257, 257, seed=seed, empty_frac=0.3, long_rows=2, long_len=60)
    b = oracle.thread_rows(A.row_ptr, nt)
    nnz = A.nnz
    ref = [0] + [int(np.searchsorted(A.row_ptr, -(-t * nnz // nt), side="left")) for t in range(1, nt)]
    ref = [min(r, A.n_rows) for r in ref] + [A.n_rows]
    assert list(b) == ref
    assert np.all(np.diff(b) >= 0)
    # the chunks cover every row once and balance the nonzeros to a row length
    maxlen = int(np.diff(A.row_ptr).max())
    for t in range(nt):
        assert abs(int(A.row_ptr[b[t + 1]] - A.row_ptr[b[t]]) - nnz / nt) <= maxlen + 1


@pytest.mark.parametrize("shape", SHAPES)
@pytest.mark.parametrize("nt", THREADS)
def test_spmv_omp_equals_plain_bit_for_bit(shape, nt):
    A = irregular(shape, 7)
    x = W.uniform(A.n_cols, 8)
    y0 = W.uniform(A.n_rows, 9)
    for alpha, beta in ALPHA_BETA:
        ref = oracle.spmv(*A.astuple(), x, alpha, beta, y0)
        # beta == 0 must not read y: start from NaN, and every row must be written
        y = y0.copy() if beta != 0.0 else np.full(A.n_rows, np.nan)
        used = oracle.spmv_omp(*A.astuple(), x, y, alpha, beta, nthreads=nt)
        assert used == (nt if nt > 0 else oracle.num_threads())
        assert np.array_equal(y, ref), (shape, nt, alpha, beta)


@pytest.mark.parametrize("nt", [1, 3, 0])
def test_spmv_omp_hamiltonian_like(nt):
    A = W.hamiltonian_like(20000, seed=31)
    x = W.uniform(A.n_rows, 32)
    y = np.full(A.n_rows, np.nan)
    oracle.spmv_omp(*A.astuple(), x, y, nthreads=nt)
    assert np.array_equal(y, oracle.spmv(*A.astuple(), x))


@pytest.mark.parametrize("shape", [(1, 1), (17, 33), (200, 150), (301, 301)])
@pytest.mark.parametrize("nt", [1, 3, 0])
def test_spmv_f32_is_the_upcast_product_rounded_once(shape, nt):
    """FP32 storage with FP64 accumulation: the products of two floats are exact in
    FP64, so the FP32 form equals the FP64 loop on the exactly upcast operands,
    rounded to float once at the end."""
    A = irregular(shape, 11)
    v32 = A.val.astype(np.float32)
    x32 = W.uniform(A.n_cols, 12).astype(np.float32)
    y32 = W.uniform(A.n_rows, 13).astype(np.float32)
    for alpha, beta in ALPHA_BETA:
        ref = oracle.spmv(A.row_ptr, A.col_idx, v32.astype(np.float64), x32.astype(np.float64), alpha, beta,
                          y32.astype(np.float64)).astype(np.float32)
        got = oracle.spmv_f32(A.row_ptr, A.col_idx, v32, x32, alpha, beta, y32, nthreads=nt)
        assert got.dtype == np.float32
        assert np.array_equal(got, ref)


def test_spmv_f32_range_extremes():
    """Products far outside the FP32 range stay exact in FP64: 1e20*1e20 = 1e40
    and 1e-25*1e-25 = 1e-50 (FP32 results round to inf and 0)."""
    rp = np.array([0, 1, 3], np.int32)
    ci = np.array([0, 0, 1], np.int32)
    v = np.array([1e20, 1e20, -1e20], np.float32)
    x = np.array([1e20, 1e20], np.float32)
    y = oracle.spmv_f32(rp, ci, v, x)
    assert np.isinf(y[0]) and y[1] == 0.0  # 1e40 overflows float; the pair cancels exactly
    v2 = np.array([1e-25, 1e-25, 1e-25], np.float32)
    x2 = np.array([1e-25, 1e-25], np.float32)
    y2 = oracle.spmv_f32(rp, ci, v2, x2)
    assert np.all(y2 == 0.0)
    ref = oracle.spmv(rp, ci, v2.astype(np.float64), x2.astype(np.float64))
    assert ref[0] == pytest.approx(1e-50, rel=1e-6) and ref[1] == pytest.approx(2e-50, rel=1e-6)


def split_literal(A, x, blocks, alpha, beta, y0):
    """Sect. 3.4 in Python loops: per block, gather the halo, then the local part
    with beta, then the nonlocal part added onto y for rows that have one."""
    y = np.array(y0, dtype=np.float64, copy=True) if beta != 0.0 else np.zeros(A.n_rows)
    for b in range(len(blocks) - 1):
        lo, hi = int(blocks[b]), int(blocks[b + 1])
        cols = sorted({int(c) for i in range(lo, hi) for c in A.col_idx[A.row_ptr[i]:A.row_ptr[i + 1]]
                       if not (lo <= c < hi)})
        halo = [float(x[c]) for c in cols]
        where = {c: h for h, c in enumerate(cols)}
        for i in range(lo, hi):
            acc = 0.0
            for k in range(A.row_ptr[i], A.row_ptr[i + 1]):
                j = int(A.col_idx[k])
                if lo <= j < hi:
                    acc = acc + float(A.val[k]) * float(x[j])
            y[i] = alpha * acc if beta == 0.0 else alpha * acc + beta * y[i]
        for i in range(lo, hi):
            acc, any_nl = 0.0, False
            for k in range(A.row_ptr[i], A.row_ptr[i + 1]):
                j = int(A.col_idx[k])
                if not (lo <= j < hi):
                    acc = acc + float(A.val[k]) * halo[where[j]]
                    any_nl = True
            if any_nl:
                y[i] = y[i] + alpha * acc
    return y


@pytest.mark.parametrize("shape", [(1, 1), (17, 17), (64, 64), (97, 97)])
@pytest.mark.parametrize("nb", [1, 2, 3, 8])
def test_spmv_split_literal_and_plain(shape, nb):
    A = irregular(shape, 21)
    x = W.uniform(A.n_cols, 22)
    y0 = W.uniform(A.n_rows, 23)
    bs = oracle.split_blocks(A.row_ptr, nb)
    for alpha, beta in ALPHA_BETA:
        got = oracle.spmv_split(*A.astuple(), x, A.n_cols, bs, alpha, beta, y0)
        assert np.array_equal(got, split_literal(A, x, bs, alpha, beta, y0))
        ref, bound = oracle.spmv(*A.astuple(), x, alpha, beta, y0, with_bound=True)
        assert np.all(np.abs(got - ref) <= 1e-13 * bound + 1e-300)


def test_spmv_split_integer_exact():
    A = W.random_csr(300, 300, seed=3, integer=True, empty_frac=0.2)
    x = W.integers(300, 4).astype(np.float64)
    bs = oracle.split_blocks(A.row_ptr, 8)
    assert np.array_equal(oracle.spmv_split(*A.astuple(), x, A.n_cols, bs), oracle.spmv(*A.astuple(), x))


@pytest.mark.parametrize("shape", [(1, 1), (64, 64), (301, 301), (200, 150)])
@pytest.mark.parametrize("nt", [1, 3, 0])
@pytest.mark.parametrize("nb", [1, 8])
def test_first_touch_node_equals_the_plain_forms(shape, nt, nb):
    """The node (first-touch copies, one chunk per thread) computes exactly the
    plain loop, the FP32-storage loop and the split form, at any thread count."""
    A = irregular(shape, 41)
    x = W.uniform(A.n_cols, 42)
    y0 = W.uniform(A.n_rows, 43)
    nd = oracle.Node(*A.astuple(), x, A.n_cols, nthreads=nt, nblocks=nb)
    assert nd.threads == (nt if nt > 0 else oracle.num_threads())
    bs = oracle.split_blocks(A.row_ptr, nb)
    assert np.array_equal(nd.block_start, bs)
    x32 = x.astype(np.float32)
    y032 = y0.astype(np.float32)
    for alpha, beta in ALPHA_BETA:
        nd.set_y(y0 if beta != 0 else np.full(A.n_rows, np.nan), y032)
        nd.spmv(alpha, beta)
        assert np.array_equal(nd.get_y()[0], oracle.spmv(*A.astuple(), x, alpha, beta, y0))
        nd.set_y(y0 if beta != 0 else np.full(A.n_rows, np.nan), y032)
        nd.spmv_split(alpha, beta)
        assert np.array_equal(nd.get_y()[0], oracle.spmv_split(*A.astuple(), x, A.n_cols, bs, alpha, beta, y0))
        nd.set_y(None, y032)
        nd.spmv_f32(alpha, beta)
        ref32 = oracle.spmv_f32(A.row_ptr, A.col_idx, A.val.astype(np.float32), x32, alpha, beta, y032)
        assert np.array_equal(nd.get_y()[1], ref32)
    nd.close()


def test_first_touch_node_hamiltonian_like():
    A = W.hamiltonian_like(30000, seed=51)
    x = W.uniform(A.n_rows, 52)
    nd = oracle.Node(*A.astuple(), x, A.n_cols, nthreads=0, nblocks=8)
    nd.spmv()
    y, _ = nd.get_y()
    assert np.array_equal(y, oracle.spmv(*A.astuple(), x))
    nd.spmv_split()
    ys, _ = nd.get_y()
    assert np.array_equal(ys, oracle.spmv_split(*A.astuple(), x, A.n_cols, nd.block_start))
    _, bound = oracle.spmv(*A.astuple(), x, with_bound=True)
    assert np.all(np.abs(ys - y) <= 1e-13 * bound)
    nd.close()
