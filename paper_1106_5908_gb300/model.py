"""Node-level code-balance model of the paper and the GPU byte counts built on it.

Eq. 1 (Sect. 1.2): per inner-loop iteration of Listing 1 the CRS kernel moves
8 bytes of ``val``, 4 bytes of ``col_idx``, 16/N_nzr bytes for the update of the
result (write-allocate plus evict) and at least 8/N_nzr bytes for the right-hand
side, plus kappa extra bytes for every further load of it, for 2 flops:

    B_CRS = (12 + 24/N_nzr + kappa)/2 = 6 + 12/N_nzr + kappa/2   bytes/flop.

Eq. 2 (Sect. 3.4): the split (local/nonlocal) form writes the result twice, adding
16/N_nzr bytes per iteration:

    B_CRS^split = 6 + 20/N_nzr + kappa/2                         bytes/flop.

kappa follows from a measured bandwidth and performance (Sect. 2):
kappa = 2*(BW/P - 6 - 12/N_nzr).  These are host-side reporting helpers.

The GPU byte counts are the algorithmic traffic of one launch: every byte of the
operands the operation must touch once (int32 row_ptr included, which the paper
omits), with no write-allocate term (GPU stores do not read the line first).
"""
from __future__ import annotations


def b_crs(nnzr: float, kappa: float = 0.0) -> float:
    """Eq. 1: code balance of the CRS spMVM in bytes per flop."""
    return 6.0 + 12.0 / nnzr + kappa / 2.0


def b_split(nnzr: float, kappa: float = 0.0) -> float:
    """Eq. 2: code balance of the split (local + nonlocal) spMVM."""
    return 6.0 + 20.0 / nnzr + kappa / 2.0


def max_performance(bandwidth: float, nnzr: float, kappa: float = 0.0) -> float:
    """Upper performance limit (flop/s in the unit of ``bandwidth``/byte) from a
    memory bandwidth and the code balance, as used in Sect. 2."""
    return bandwidth / b_crs(nnzr, kappa)


def kappa_from(bandwidth: float, performance: float, nnzr: float) -> float:
    """Sect. 2: the kappa that makes B_CRS equal the measured bytes per flop."""
    return 2.0 * (bandwidth / performance - 6.0 - 12.0 / nnzr)


def rhs_loads(kappa: float, nnzr: float) -> float:
    """How many times the right-hand side is loaded from memory per spMVM: once,
    plus kappa*N_nzr/8 (kappa grows by 8/N_nzr per extra load, Sect. 1.2)."""
    return 1.0 + kappa * nnzr / 8.0


def split_penalty(nnzr: float, kappa: float = 0.0) -> float:
    """Relative code-balance increase of the split form over the plain one."""
    return b_split(nnzr, kappa) / b_crs(nnzr, kappa) - 1.0


# ---------------------------------------------------------------------------
# GPU algorithmic byte counts (one launch)
# ---------------------------------------------------------------------------

def bytes_plain(n_rows: int, n_cols: int, nnz: int, val_bytes: int = 8, x_bytes: int = 8,
                y_bytes: int = 8, beta_nonzero: bool = False) -> int:
    """val + col_idx per entry, row_ptr, x read once, y written once (and read
    once when beta != 0)."""
    b = (val_bytes + 4) * nnz + 4 * (n_rows + 1) + x_bytes * n_cols + y_bytes * n_rows
    if beta_nonzero:
        b += y_bytes * n_rows
    return int(b)


def bytes_split_vector(n_rows: int, n_cols: int, nnz: int, total_halo: int,
                       beta_nonzero: bool = False) -> int:
    """Vector mode: plain FP64 bytes, plus x copied into the extended vector
    (read + write) and the halo traffic (map read, gathered x read, halo write,
    halo read: 4 + 8 + 8 + 8 bytes per halo entry); y is written once."""
    return int(bytes_plain(n_rows, n_cols, nnz, beta_nonzero=beta_nonzero) + 16 * n_rows + 28 * total_halo)


def bytes_split(n_rows: int, n_cols: int, nnz: int, total_halo: int,
                beta_nonzero: bool = False) -> int:
    """Plain FP64 bytes plus the second pass over y (read + write, Eq. 2) and the
    second row_ptr, plus the halo traffic: map read, gathered x read, halo write,
    halo read (4 + 8 + 8 + 8 bytes per halo entry)."""
    return int(bytes_plain(n_rows, n_cols, nnz, beta_nonzero=beta_nonzero)
               + 16 * n_rows + 4 * (n_rows + 1) + 28 * total_halo)


def bytes_spmm(n_rows: int, n_cols: int, nnz: int, nrhs: int,
               beta_nonzero: bool = False) -> int:
    """Block vectors: the matrix once, X read once and Y written once (8*nrhs each
    per row)."""
    b = 12 * nnz + 4 * (n_rows + 1) + 8 * nrhs * (n_cols + n_rows)
    if beta_nonzero:
        b += 8 * nrhs * n_rows
    return int(b)


def bytes_backward(n_rows: int, n_cols: int, nnz: int, grad_x: bool = True,
                   grad_val: bool = True, val_bytes: int = 8, vec_bytes: int = 8) -> int:
    """grad_x through the transposed CRS (colT + perm per entry, val read through
    perm, rowT_ptr, g read once, grad_x written once) and grad_val (col_idx read,
    row_ptr, x and g read once, grad_val written); val_bytes / vec_bytes 4 for
    FP32 storage."""
    b = 0
    if grad_x:
        b += (4 + 4 + val_bytes) * nnz + 4 * (n_cols + 1) + vec_bytes * (n_rows + n_cols)
    if grad_val:
        b += (4 + val_bytes) * nnz + 4 * (n_rows + 1) + vec_bytes * (n_cols + n_rows)
    return int(b)


def bytes_symmetric(n: int, nnz_upper: int, nnz_strict: int, implementation: bool = False) -> int:
    """Symmetric CRS (Sect. 1.3.1): the upper triangle with the diagonal read once
    (value + column index per stored entry), row_ptr, x read once, y written once
    -- the single-pass scheme whose traffic the paper expects to halve.  With
    ``implementation`` the two passes this library runs: the upper triangle's
    row sums, then the transposed strictly upper part (row_ptr, row index and
    value position per entry, the value read through that position, x read
    again, y read and written again)."""
    b = 12 * nnz_upper + 4 * (n + 1) + 8 * n + 8 * n
    if implementation:
        b += (4 + 4 + 8) * nnz_strict + 4 * (n + 1) + 8 * n + 16 * n
    return int(b)


def flops(nnz: int, nrhs: int = 1) -> int:
    """Two flops per entry and right-hand side (Sect. 1.2)."""
    return int(2 * nnz * nrhs)
