"""Seeded synthetic CRS matrices and vectors shaped like the paper's workloads.

This module only draws inputs.  It contains none of the spMVM arithmetic, imports
neither the oracle nor the CUDA binding, and is the one module both sides share.
All generators use numpy's PCG64 (``np.random.default_rng(seed)``) and return
0-based CRS arrays ``(row_ptr int32, col_idx int32, val float64)`` with columns
sorted within each row unless stated otherwise.

Stand-ins for the paper's matrices (Sect. 1.3.1), which are not available here:
  * ``hamiltonian_like`` for the HMeP Holstein-Hubbard matrix (symmetric, banded
    plus scattered entries, N_nzr around 13-15);
  * ``laplace3d`` for the sAMG Poisson matrix (N_nzr about 7);
  * ``stencil27`` for the higher-N_nzr regime (UHBR has N_nzr about 123, not
    reproduced).
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np

# Fixed seeds of the synthetic workloads.
SEED_LAPLACE2D_X = 1101
SEED_LAPLACE2D_XINT = 1102
SEED_HAMILTONIAN = 2201
SEED_HAMILTONIAN_X = 2202
SEED_POISSON7_B = 3301
SEED_BLOCK_X = 4401
SEED_BATCH = 4402
SEED_STENCIL27_VAL = 5501
SEED_STENCIL27_X = 5502
SEED_STENCIL27_G = 5503
SEED_FP32_RANGE = 7701


@dataclass
class CRS:
    row_ptr: np.ndarray  # int32, n_rows + 1
    col_idx: np.ndarray  # int32, nnz
    val: np.ndarray      # float64, nnz
    n_cols: int

    @property
    def n_rows(self) -> int:
        return int(self.row_ptr.size - 1)

    @property
    def nnz(self) -> int:
        return int(self.row_ptr[-1])

    def astuple(self):
        return self.row_ptr, self.col_idx, self.val


def _row_ptr_from_counts(counts: np.ndarray) -> np.ndarray:
    rp = np.zeros(counts.size + 1, np.int64)
    np.cumsum(counts, out=rp[1:])
    return rp.astype(np.int32)


def _stencil(shape, offsets, diag_value, off_value, vals=None) -> CRS:
    """Truncated (Dirichlet) stencil on a lexicographic grid, first axis fastest.
    ``offsets`` are tuples in the order of ``shape`` listed so that the linear
    column offset increases; entries outside the grid are dropped."""
    dims = len(shape)
    n = int(np.prod(shape))
    idx = np.arange(n, dtype=np.int64)
    coords = []
    rem = idx
    for d in range(dims):
        coords.append(rem % shape[d])
        rem = rem // shape[d]
    strides = [int(np.prod(shape[:d])) for d in range(dims)]
    cols = np.full((n, len(offsets)), -1, dtype=np.int64)
    for m, off in enumerate(offsets):
        ok = np.ones(n, bool)
        lin = idx.copy()
        for d in range(dims):
            c = coords[d] + off[d]
            ok &= (c >= 0) & (c < shape[d])
            lin += off[d] * strides[d]
        cols[ok, m] = lin[ok]
    mask = cols >= 0
    counts = mask.sum(axis=1)
    col_idx = cols[mask].astype(np.int32)  # row-major flatten keeps rows, columns ascend
    if vals is None:
        is_diag = np.zeros((n, len(offsets)), bool)
        for m, off in enumerate(offsets):
            if all(o == 0 for o in off):
                is_diag[:, m] = True
        val = np.where(is_diag[mask], diag_value, off_value).astype(np.float64)
    else:
        val = vals(int(mask.sum()))
    return CRS(_row_ptr_from_counts(counts), col_idx, val, n)


def _sorted_offsets(dims, radius_set):
    offs = [o for o in radius_set]
    # order by linear offset: last axis most significant
    def key(o):
        return tuple(reversed(o))
    return sorted(offs, key=key)


def laplace2d(nx: int, ny: int | None = None) -> CRS:
    """2D 5-point Laplacian, diagonal 4, off-diagonals -1, Dirichlet boundary
    (truncated stencil), x fastest."""
    ny = nx if ny is None else ny
    offs = [(0, -1), (-1, 0), (0, 0), (1, 0), (0, 1)]
    return _stencil((nx, ny), _sorted_offsets(2, offs), 4.0, -1.0)


def laplace3d(n: int) -> CRS:
    """3D 7-point Laplacian on an n^3 grid, diagonal 6, off-diagonals -1."""
    offs = [(0, 0, 0), (-1, 0, 0), (1, 0, 0), (0, -1, 0), (0, 1, 0), (0, 0, -1), (0, 0, 1)]
    return _stencil((n, n, n), _sorted_offsets(3, offs), 6.0, -1.0)


def stencil27(n: int, seed: int = SEED_STENCIL27_VAL) -> CRS:
    """27-point pattern on an n^3 grid (diagonal included), values N(0,1), not
    symmetric."""
    offs = [(a, b, c) for a in (-1, 0, 1) for b in (-1, 0, 1) for c in (-1, 0, 1)]
    rng = np.random.default_rng(seed)
    return _stencil((n, n, n), _sorted_offsets(3, offs), 0.0, 0.0,
                    vals=lambda m: rng.standard_normal(m))


def _distinct_draw(rng, avail, counts, kmax):
    """For every row r draw counts[r] distinct offsets from [0, avail[r]) with
    Floyd's subset algorithm, vectorised over rows.  Returns an int64 array of
    shape (rows, kmax) holding the offsets sorted ascending, padded with -1."""
    n = avail.size
    counts = np.minimum(counts, avail)
    out = np.full((n, kmax), -1, np.int64)
    for m in range(kmax):
        act = np.nonzero(counts > m)[0]
        if act.size == 0:
            break
        # Floyd: for j = avail-k+m, draw t in [0, j]; take j if t was drawn already
        j = avail[act] - counts[act] + m
        t = rng.integers(0, j + 1, dtype=np.int64)
        seen = (out[act, :m] == t[:, None]).any(axis=1) if m else np.zeros(act.size, bool)
        out[act, m] = np.where(seen, j, t)
    big = np.iinfo(np.int64).max
    srt = np.sort(np.where(out < 0, big, out), axis=1)
    return np.where(srt == big, -1, srt)


def hamiltonian_like(n: int, seed: int = SEED_HAMILTONIAN, band: int = 64,
                     mean_len: float = 6.0, min_len: int = 2, max_len: int = 16) -> CRS:
    """Symmetric Hamiltonian-like matrix (stand-in for HMeP).

    Upper-triangle row length l_i = clip(Poisson(mean_len), min_len, max_len);
    ceil(l_i/2) distinct columns from (i, min(i+band, n-1)] and floor(l_i/2)
    distinct columns from [i+band+1, n); a shortfall in one range moves to the
    other; values N(0,1).  The upper part is mirrored to the lower triangle and a
    N(0,1) diagonal is added; columns are sorted within rows."""
    rng = np.random.default_rng(seed)
    i = np.arange(n, dtype=np.int64)
    L = np.clip(rng.poisson(mean_len, n), min_len, max_len).astype(np.int64)
    near_avail = np.minimum(band, n - 1 - i)
    far_avail = np.maximum(0, n - (i + band + 1))
    n_near = (L + 1) // 2
    n_far = L // 2
    over = np.maximum(0, n_near - near_avail)
    n_near -= over
    n_far += over
    over = np.maximum(0, n_far - far_avail)
    n_far -= over
    n_near = np.minimum(near_avail, n_near + over)
    near = _distinct_draw(rng, near_avail, n_near, max_len)
    far = _distinct_draw(rng, far_avail, n_far, max_len)
    # upper part of every row, columns ascending (near < far), row-major order
    up = np.concatenate([np.where(near >= 0, near + i[:, None] + 1, -1),
                         np.where(far >= 0, far + i[:, None] + band + 1, -1)], axis=1)
    keep = up >= 0
    n_up = keep.sum(axis=1)
    up_c = up[keep]
    up_r = np.repeat(i, n_up)
    up_v = rng.standard_normal(up_c.size)
    diag_v = rng.standard_normal(n)
    # mirror to the lower triangle, add the diagonal; scipy's COO -> CSR conversion
    # is a counting sort by row, after which columns are sorted within rows
    import scipy.sparse as sp
    rows = np.concatenate([up_r, up_c, i]).astype(np.int32)
    cols = np.concatenate([up_c, up_r, i]).astype(np.int32)
    vals = np.concatenate([up_v, up_v, diag_v])
    m = sp.csr_matrix((vals, (rows, cols)), shape=(n, n))
    m.sort_indices()
    return CRS(m.indptr.astype(np.int32), m.indices.astype(np.int32),
               m.data.astype(np.float64), n)


def random_csr(n_rows: int, n_cols: int, seed: int, max_len: int = 8, empty_frac: float = 0.2,
               dup_frac: float = 0.1, sort_cols: bool = False, integer: bool = False,
               long_rows: int = 0, long_len: int = 0) -> CRS:
    """Small irregular CRS for tests: some empty rows, repeated (row, col) entries,
    unsorted columns; optionally integer values in [-4, 4] and a few long rows."""
    rng = np.random.default_rng(seed)
    lens = rng.integers(0, max_len + 1, n_rows)
    lens[rng.random(n_rows) < empty_frac] = 0
    if long_rows and n_rows:
        pick = rng.choice(n_rows, size=min(long_rows, n_rows), replace=False)
        lens[pick] = long_len
    if n_cols == 0:
        lens[:] = 0
    nnz = int(lens.sum())
    cols = rng.integers(0, max(n_cols, 1), nnz) if nnz else np.zeros(0, np.int64)
    # plant repeats: copy a column from earlier in the same row
    rp = _row_ptr_from_counts(lens).astype(np.int64)
    if nnz:
        row_of = np.repeat(np.arange(n_rows), lens)
        pos = np.arange(nnz) - rp[row_of]
        cand = (pos > 0) & (rng.random(nnz) < dup_frac)
        cols[cand] = cols[np.nonzero(cand)[0] - 1]
        if sort_cols:
            order = np.lexsort((cols, row_of))
            cols = cols[order]
    if integer:
        val = rng.integers(-4, 5, nnz).astype(np.float64)
    else:
        val = rng.standard_normal(nnz)
    return CRS(rp.astype(np.int32), cols.astype(np.int32), val, n_cols)


def uniform(n: int, seed: int, lo: float = -1.0, hi: float = 1.0, shape=None) -> np.ndarray:
    rng = np.random.default_rng(seed)
    return rng.uniform(lo, hi, n if shape is None else shape)


def integers(n: int, seed: int, lo: int = -8, hi: int = 8) -> np.ndarray:
    rng = np.random.default_rng(seed)
    return rng.integers(lo, hi + 1, n).astype(np.float64)


def truncated_laplace2d(n: int) -> CRS:
    """5-point Laplacian on the floor(sqrt n) x ceil(n/floor(sqrt n)) grid, cut to
    its leading n x n block (rows and columns >= n dropped)."""
    nx = max(1, int(math.isqrt(n)))
    ny = -(-n // nx)
    full = laplace2d(nx, ny)
    rp = full.row_ptr[: n + 1].astype(np.int64)
    cols = full.col_idx[: rp[-1]]
    vals = full.val[: rp[-1]]
    keep = cols < n
    row_of = np.repeat(np.arange(n), np.diff(rp))
    counts = np.bincount(row_of[keep], minlength=n)
    return CRS(_row_ptr_from_counts(counts), cols[keep].astype(np.int32), vals[keep], n)


def batch_sizes(count: int = 256, seed: int = SEED_BATCH, lo: int = 1000, hi: int = 200000):
    rng = np.random.default_rng(seed)
    return rng.integers(lo, hi + 1, count)


def batch_matrix(m: int, n: int, seed: int = SEED_BATCH) -> CRS:
    """Matrix m of the uneven batch: even m a truncated 2D 5-point Laplacian, odd m
    a Hamiltonian-like pattern, both of order n."""
    if m % 2 == 0:
        return truncated_laplace2d(int(n))
    return hamiltonian_like(int(n), seed=seed * 1000 + m)


# Orderings for the ordering study (the paper's RCM remark, Sect. 2): the
# matrix P A P^T, where row/column i of the result is row/column order[i] of A.
SEED_ORDER_RANDOM = 6601


def rcm_order(A: CRS) -> np.ndarray:
    """Reverse Cuthill-McKee order of the (symmetric) pattern of A."""
    import scipy.sparse as sp
    from scipy.sparse.csgraph import reverse_cuthill_mckee
    M = sp.csr_matrix((np.ones(A.nnz, np.int8), A.col_idx, A.row_ptr), shape=(A.n_rows, A.n_cols))
    return np.asarray(reverse_cuthill_mckee(M, symmetric_mode=True), dtype=np.int64)


def random_order(n: int, seed: int = SEED_ORDER_RANDOM) -> np.ndarray:
    return np.random.default_rng(seed).permutation(n)


def permute_symmetric(A: CRS, order: np.ndarray) -> CRS:
    """P A P^T: entry (i, j) of the result is entry (order[i], order[j]) of A;
    columns sorted within each row."""
    import scipy.sparse as sp
    M = sp.csr_matrix((A.val, A.col_idx, A.row_ptr), shape=(A.n_rows, A.n_cols))
    order = np.asarray(order, dtype=np.int64)
    P = M[order][:, order].tocsr()
    P.sort_indices()
    return CRS(P.indptr.astype(np.int32), P.indices.astype(np.int32), P.data.astype(A.val.dtype), A.n_cols)


def bandwidth(A: CRS) -> int:
    """max |i - j| over the entries (i, j)."""
    rows = np.repeat(np.arange(A.n_rows), np.diff(A.row_ptr.astype(np.int64)))
    return int(np.abs(rows - A.col_idx).max()) if A.nnz else 0


# Shapes of the five synthetic configurations.
LAPLACE2D_GRID = 256          # 2D 5-point, N = 65,536
HAMILTONIAN_N = 4_194_304       # Hamiltonian-like, N = 4,194,304
POISSON7_GRID = 160          # 3D 7-point, N = 4,096,000
BLOCK_NRHS = (1, 4, 8, 16, 32)
BATCH_COUNT = 256
STENCIL27_GRID = 128          # 3D 27-point, N = 2,097,152
STENCIL27_FD_GRID = 16


def fp32_range_case(seed: int = SEED_FP32_RANGE, n_normal: int = 3000, n_wild: int = 400,
                    long_len: int = 3000, special: bool = True):
    """FP32-stored values and vector whose products leave FP32's range, mixed
    into ordinary rows (for the FP32-storage parity tests).  Returns (CRS with
    float32 values, x float32).

    x holds special values at fixed positions (1e20, -1e20, 1e-25, -1e-25, 1,
    1.8e19, 2^-50, 2^-51, a subnormal, 0, 3e38, 1.5, and with ``special`` inf and
    NaN); designed rows reach products above FLT_MAX (alone, cancelling, and as a
    sum of two products below it), products far below the smallest subnormal
    (alone, cancelling, next to a product of one), products on either side of
    2^-100, zero values and zero x, and inf/NaN operands; ``n_wild`` rows draw
    values and x entries with log-uniform magnitudes over the whole FP32 range
    and ``n_wild/2`` rows over [2^-149, 2^-50] only (every product below 2^-100);
    one row has ``long_len`` entries of the first kind; ``n_normal`` rows are N(0,1) values on
    U[-1,1] entries.  The rows are shuffled, so chunks and slices mix them."""
    rng = np.random.default_rng(seed)
    spec = [1e20, -1e20, 1e-25, -1e-25, 1.0, 1.8e19, 2.0 ** -50, 2.0 ** -51, 1e-40, 0.0, 3e38, 1.5]
    if special:
        spec += [np.inf, np.nan]
    n_spec = len(spec)
    n_cols = 4096

    def logu(k, lo=-149.0, hi=127.0):
        mag = np.exp2(rng.uniform(lo, hi, k))
        return (mag * np.where(rng.random(k) < 0.5, -1.0, 1.0)).astype(np.float32)

    x = np.empty(n_cols, np.float32)
    x[:n_spec] = np.array(spec, np.float64).astype(np.float32)
    wild_lo, wild_hi, tiny_hi = n_spec, 1024, 1280
    x[wild_lo:wild_hi] = logu(wild_hi - wild_lo)
    x[wild_hi:tiny_hi] = logu(tiny_hi - wild_hi, -149.0, -50.0)
    x[tiny_hi:] = rng.uniform(-1.0, 1.0, n_cols - tiny_hi).astype(np.float32)
    rows = [
        [(0, 1e20)], [(0, 1e20), (1, 1e20)], [(2, 1e-25)], [(2, 1e-25), (3, 1e-25)],
        [(4, 1.0), (2, 1e-25)], [(5, 1.8e19), (5, 1.8e19)], [(6, 2.0 ** -50)], [(7, 2.0 ** -50)],
        [(8, 1.0)], [(9, 1e-30)], [(2, 0.0)], [(10, 3e38), (10, -3e38)], [(11, 1.5)] * 20, [],
        [(4, 1.0), (0, 1e20), (1, 1e20), (4, -1.0)], [(8, 1e-5), (2, 1e-25), (6, 2.0 ** -60)],
    ]
    if special:
        rows += [[(12, 1.0)], [(12, 0.0)], [(13, 2.0)], [(4, 1.0), (12, -1.0), (12, 1.0)]]
    for _ in range(n_wild):
        k = int(rng.integers(1, 41))
        cols = rng.integers(wild_lo, wild_hi, k)
        rows.append(list(zip(cols.tolist(), logu(k).tolist())))
    for _ in range(n_wild // 2):  # every product below 2^-100
        k = int(rng.integers(1, 41))
        cols = rng.integers(wild_hi, tiny_hi, k)
        rows.append(list(zip(cols.tolist(), logu(k, -149.0, -50.0).tolist())))
    cols = rng.integers(wild_lo, wild_hi, long_len)
    rows.append(list(zip(cols.tolist(), logu(long_len).tolist())))
    for _ in range(n_normal):
        k = int(rng.integers(1, 25))
        cols = rng.integers(tiny_hi, n_cols, k)
        rows.append(list(zip(cols.tolist(), rng.standard_normal(k).tolist())))
    order = rng.permutation(len(rows))
    rows = [rows[i] for i in order]
    counts = np.array([len(r) for r in rows], np.int64)
    rp = _row_ptr_from_counts(counts)
    col = np.array([c for r in rows for c, _ in r], np.int32)
    val = np.array([v for r in rows for _, v in r], np.float64).astype(np.float32)
    return CRS(rp, col, val, n_cols), x


def column_heavy_csr(n_rows: int, n_cols: int, seed: int, dense: int = 1, medium: int = 50,
                     medium_len: int = 2000, max_len: int = 6) -> CRS:
    """Irregular CRS with long columns (for the transposed build): ``dense``
    columns with an entry in every row, ``medium`` columns with about
    ``medium_len`` entries each (rows drawn at random), and up to ``max_len``
    random other entries per row; columns unsorted within rows, N(0,1) values."""
    rng = np.random.default_rng(seed)
    dense_cols = rng.choice(n_cols, size=min(dense, n_cols), replace=False)
    med_cols = rng.choice(n_cols, size=min(medium, n_cols), replace=False)
    per_row = [[] for _ in range(n_rows)]
    for c in dense_cols.tolist():
        for i in range(n_rows):
            per_row[i].append(c)
    for c in med_cols.tolist():
        for i in rng.integers(0, n_rows, min(medium_len, n_rows)).tolist():
            per_row[i].append(c)
    lens = rng.integers(0, max_len + 1, n_rows)
    for i in range(n_rows):
        per_row[i].extend(rng.integers(0, n_cols, int(lens[i])).tolist())
        rng.shuffle(per_row[i])
    counts = np.array([len(r) for r in per_row], np.int64)
    rp = _row_ptr_from_counts(counts)
    col = np.array([c for r in per_row for c in r], np.int32)
    return CRS(rp, col, rng.standard_normal(col.size), n_cols)


def upper_triangle(A: CRS) -> CRS:
    """The entries of A with col >= row (the upper triangle with the diagonal),
    row by row in A's order: the stored form of a symmetric matrix."""
    rows = np.repeat(np.arange(A.n_rows, dtype=np.int64), np.diff(A.row_ptr.astype(np.int64)))
    keep = A.col_idx[: A.nnz] >= rows
    counts = np.bincount(rows[keep], minlength=A.n_rows)
    return CRS(_row_ptr_from_counts(counts), A.col_idx[: A.nnz][keep].copy(), A.val[: A.nnz][keep].copy(), A.n_cols)


def random_symmetric_upper(n: int, seed: int, max_len: int = 8, integer: bool = False, empty_frac: float = 0.1) -> CRS:
    """Upper triangle with diagonal of a random symmetric n x n matrix: some rows
    without a diagonal, some empty, repeated (row, col) entries, unsorted columns."""
    rng = np.random.default_rng(seed)
    per_row = []
    for i in range(n):
        k = int(rng.integers(0, max_len + 1)) if rng.random() >= empty_frac else 0
        cols = list(rng.integers(i, n, k)) if n - i > 0 else []
        if cols and rng.random() < 0.2:
            cols.append(cols[0])  # a repeated entry
        rng.shuffle(cols)
        per_row.append(cols)
    counts = np.array([len(r) for r in per_row], np.int64)
    col = np.array([c for r in per_row for c in r], np.int32)
    val = rng.integers(-4, 5, col.size).astype(np.float64) if integer else rng.standard_normal(col.size)
    return CRS(_row_ptr_from_counts(counts), col, val, n)
