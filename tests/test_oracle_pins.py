"""Pins of the oracle against things other than itself: dense and library
products, closed forms of the stencil operators, eigenpairs, invariants, exact
integer arithmetic and brute force on tiny inputs.  CPU only."""
import math

import numpy as np
import pytest
import scipy.sparse as sp

import oracle
from paper_1106_5908_gb300 import workloads as W


def dense_of(A: W.CRS) -> np.ndarray:
    """Dense matrix assembled entry by entry (repeats summed) with np.add.at."""
    D = np.zeros((A.n_rows, A.n_cols))
    rows = np.repeat(np.arange(A.n_rows), np.diff(A.row_ptr))
    np.add.at(D, (rows, A.col_idx[: A.nnz]), A.val[: A.nnz])
    return D


def within(y, ref, bound, rel):
    return np.all(np.abs(y - ref) <= rel * bound + 1e-300)


CASES = [(0, 0), (1, 1), (1, 5), (5, 1), (7, 7), (17, 33), (64, 64), (64, 40), (200, 150)]


@pytest.mark.parametrize("shape", CASES)
@pytest.mark.parametrize("seed", [1, 2, 3])
def test_spmv_vs_dense_and_scipy(shape, seed):
    n_rows, n_cols = shape
    A = W.random_csr(n_rows, n_cols, seed=seed)
    x = W.uniform(n_cols, seed + 100)
    y0 = W.uniform(n_rows, seed + 200)
    for alpha, beta in [(1.0, 0.0), (-0.5, 1.0), (2.0, -3.0), (0.0, 1.5), (1.0, 1.0)]:
        y, bound = oracle.spmv(*A.astuple(), x, alpha, beta, y0, with_bound=True)
        ref = alpha * (dense_of(A) @ x) + (beta * y0 if beta != 0 else 0.0)
        assert y.shape == (n_rows,)
        assert within(y, ref, bound, 1e-13)
        if n_rows and n_cols:
            m = sp.csr_matrix((A.val, A.col_idx, A.row_ptr), shape=(n_rows, n_cols))
            assert within(y, alpha * (m @ x) + (beta * y0 if beta else 0.0), bound, 1e-13)


def test_beta_zero_does_not_read_y():
    A = W.random_csr(30, 30, seed=4)
    x = W.uniform(30, 5)
    y0 = np.full(30, np.nan)
    y = oracle.spmv(*A.astuple(), x, 1.0, 0.0, y0)
    assert np.all(np.isfinite(y))


def test_empty_rows_give_beta_y():
    A = W.random_csr(50, 20, seed=6, empty_frac=0.5)
    x = W.uniform(20, 7)
    y0 = W.uniform(50, 8)
    y = oracle.spmv(*A.astuple(), x, 3.0, 0.25, y0)
    empty = np.diff(A.row_ptr) == 0
    assert empty.any()
    assert np.array_equal(y[empty], 0.25 * y0[empty])


def test_one_based_listing_reading():
    """Listing 1 is Fortran with 1-based row_ptr/col_idx and C(i) = C(i) + ...; the
    0-based ABI with alpha = beta = 1 is the same operation."""
    A = W.random_csr(12, 9, seed=9, integer=True)
    x = W.integers(9, 10)
    C = W.integers(12, 11)
    row_ptr1 = [int(v) + 1 for v in A.row_ptr]        # 1-based offsets
    col1 = [int(c) + 1 for c in A.col_idx]             # 1-based columns
    B1 = [None] + list(x)                              # B(1..n)
    C1 = [None] + list(C)
    for i in range(1, A.n_rows + 1):
        for j in range(row_ptr1[i - 1], row_ptr1[i]):  # row_ptr(i) .. row_ptr(i+1)-1
            C1[i] = C1[i] + A.val[j - 1] * B1[col1[j - 1]]
    y = oracle.spmv(*A.astuple(), x, 1.0, 1.0, C)
    assert np.array_equal(y, np.array(C1[1:], dtype=np.float64))


def grid_coords(shape):
    n = int(np.prod(shape))
    idx = np.arange(n)
    out = []
    for s in shape:
        out.append(idx % s)
        idx = idx // s
    return out


@pytest.mark.parametrize("nx,ny", [(1, 1), (2, 3), (5, 5), (16, 9), (33, 20)])
def test_laplace2d_closed_forms(nx, ny):
    A = W.laplace2d(nx, ny)
    ix, iy = grid_coords((nx, ny))
    nb = (ix > 0).astype(int) + (ix < nx - 1) + (iy > 0) + (iy < ny - 1)
    # x = 1: row sum = 4 - number of neighbours
    y = oracle.spmv(*A.astuple(), np.ones(A.n_rows))
    assert np.array_equal(y, 4.0 - nb)
    interior = (ix > 0) & (ix < nx - 1) & (iy > 0) & (iy < ny - 1)
    # linear functions are in the kernel of the interior stencil
    for f in (ix.astype(float), iy.astype(float), 3.0 * ix - 2.0 * iy + 1.0):
        y = oracle.spmv(*A.astuple(), f)
        assert np.array_equal(y[interior], np.zeros(interior.sum()))
    # x = i^2 along one axis gives -2 inside
    y = oracle.spmv(*A.astuple(), ix.astype(float) ** 2)
    assert np.array_equal(y[interior], np.full(interior.sum(), -2.0))


@pytest.mark.parametrize("n", [1, 2, 6, 11])
def test_laplace3d_closed_forms(n):
    A = W.laplace3d(n)
    ix, iy, iz = grid_coords((n, n, n))
    nb = sum(((c > 0).astype(int) + (c < n - 1)) for c in (ix, iy, iz))
    y = oracle.spmv(*A.astuple(), np.ones(A.n_rows))
    assert np.array_equal(y, 6.0 - nb)
    interior = np.ones(A.n_rows, bool)
    for c in (ix, iy, iz):
        interior &= (c > 0) & (c < n - 1)
    y = oracle.spmv(*A.astuple(), (ix + 2 * iy - iz).astype(float))
    assert np.array_equal(y[interior], np.zeros(interior.sum()))
    y = oracle.spmv(*A.astuple(), iz.astype(float) ** 2)
    assert np.array_equal(y[interior], np.full(interior.sum(), -2.0))


@pytest.mark.parametrize("dims,n,ks", [(2, 12, (1, 1)), (2, 12, (3, 7)), (3, 8, (1, 2, 5)),
                                       (3, 8, (8, 8, 8))])
def test_dirichlet_eigenpairs(dims, n, ks):
    A = W.laplace2d(n) if dims == 2 else W.laplace3d(n)
    coords = grid_coords((n,) * dims)
    v = np.ones(A.n_rows)
    lam = 0.0
    for c, k in zip(coords, ks):
        v *= np.sin(math.pi * k * (c + 1) / (n + 1))
        lam += 2.0 - 2.0 * math.cos(math.pi * k / (n + 1))
    y = oracle.spmv(*A.astuple(), v)
    assert np.max(np.abs(y - lam * v)) <= 1e-13 * max(1.0, np.max(np.abs(lam * v)))


def test_stencil27_row_sums():
    A = W.stencil27(6, seed=3)
    assert A.n_rows == 216
    assert A.nnz == (3 * 6 - 2) ** 3  # (3n-2)^3 entries on an n^3 grid
    y = oracle.spmv(*A.astuple(), np.ones(A.n_rows))
    rows = np.repeat(np.arange(A.n_rows), np.diff(A.row_ptr))
    ref = np.bincount(rows, weights=A.val, minlength=A.n_rows)
    _, bound = oracle.spmv(*A.astuple(), np.ones(A.n_rows), with_bound=True)
    assert within(y, ref, bound, 1e-14)


@pytest.mark.parametrize("n", [200, 3000])
def test_symmetry_invariant(n):
    A = W.hamiltonian_like(n, seed=n)
    x = W.uniform(n, 1)
    z = W.uniform(n, 2)
    yx = oracle.spmv(*A.astuple(), x)
    yz = oracle.spmv(*A.astuple(), z)
    lhs, rhs = z @ yx, x @ yz
    scale = np.abs(z) @ oracle.spmv(A.row_ptr, A.col_idx, np.abs(A.val), np.abs(x))
    assert abs(lhs - rhs) <= 1e-12 * scale


def test_symmetry_invariant_fails_for_nonsymmetric():
    # the invariant detects a transposed operand: it must fail on a general matrix
    A = W.stencil27(5, seed=1)
    x = W.uniform(A.n_rows, 1)
    z = W.uniform(A.n_rows, 2)
    assert abs(z @ oracle.spmv(*A.astuple(), x) - x @ oracle.spmv(*A.astuple(), z)) > 1e-6


@pytest.mark.parametrize("seed", [1, 2])
def test_integer_exact(seed):
    A = W.random_csr(300, 250, seed=seed, integer=True, max_len=20)
    x = W.integers(250, seed + 5)
    Di = np.zeros((300, 250), dtype=np.int64)
    rows = np.repeat(np.arange(300), np.diff(A.row_ptr))
    np.add.at(Di, (rows, A.col_idx), A.val.astype(np.int64))
    ref = Di @ x.astype(np.int64)
    assert np.array_equal(oracle.spmv(*A.astuple(), x), ref.astype(np.float64))
    L = W.laplace2d(40)
    xi = W.integers(L.n_rows, seed + 7)
    Dl = np.zeros((L.n_rows, L.n_rows), dtype=np.int64)
    rows = np.repeat(np.arange(L.n_rows), np.diff(L.row_ptr))
    np.add.at(Dl, (rows, L.col_idx), L.val.astype(np.int64))
    assert np.array_equal(oracle.spmv(*L.astuple(), xi), (Dl @ xi.astype(np.int64)).astype(float))


@pytest.mark.parametrize("nrhs", [1, 3, 4, 8, 32])
def test_spmm_vs_dense(nrhs):
    A = W.random_csr(70, 50, seed=nrhs)
    X = W.uniform(0, 3, shape=(50, nrhs))
    Y0 = W.uniform(0, 4, shape=(70, nrhs))
    for alpha, beta in [(1.0, 0.0), (0.5, -2.0)]:
        Y, bound = oracle.spmm(*A.astuple(), X, alpha, beta, Y0, with_bound=True)
        ref = alpha * dense_of(A) @ X + (beta * Y0 if beta else 0.0)
        assert within(Y, ref, bound, 1e-13)


@pytest.mark.parametrize("shape,sort", [((40, 30), False), ((30, 40), True), ((1, 1), False),
                                        ((0, 5), False), ((5, 0), False), ((100, 100), True)])
def test_transpose_vs_scipy(shape, sort):
    A = W.random_csr(*shape, seed=7, sort_cols=sort)
    rpt, cit, perm = oracle.transpose(A.row_ptr, A.col_idx, A.n_cols)
    assert rpt.shape == (A.n_cols + 1,) and cit.shape == (A.nnz,)
    if A.nnz:
        m = sp.csr_matrix((np.arange(1, A.nnz + 1, dtype=float), A.col_idx, A.row_ptr), shape=shape)
        t = m.tocsc()  # column-major copy: entries of a column in row order, repeats kept
        assert np.array_equal(rpt, t.indptr)
        assert np.array_equal(cit, t.indices)
        assert np.array_equal(perm + 1, t.data.astype(np.int64))
        # perm is a permutation and A^T entries reference their own column
        assert np.array_equal(np.sort(perm), np.arange(A.nnz))
        rows = np.repeat(np.arange(A.n_cols), np.diff(rpt))
        assert np.array_equal(A.col_idx[perm], rows)
        # within a row of A^T, original positions increase
        for j in range(A.n_cols):
            assert np.all(np.diff(perm[rpt[j]:rpt[j + 1]]) > 0)


def test_transpose_twice_is_identity():
    A = W.random_csr(60, 45, seed=3, sort_cols=True, dup_frac=0.0)
    # drop repeats so the pattern is a set
    m = sp.csr_matrix((A.val, A.col_idx, A.row_ptr), shape=(60, 45))
    m.sum_duplicates()
    rp, ci = m.indptr.astype(np.int32), m.indices.astype(np.int32)
    rpt, cit, _ = oracle.transpose(rp, ci, 45)
    rp2, ci2, _ = oracle.transpose(rpt, cit, 60)
    assert np.array_equal(rp2, rp) and np.array_equal(ci2, ci)


@pytest.mark.parametrize("seed", [1, 2])
def test_backward_vs_dense_and_fd(seed):
    A = W.random_csr(45, 35, seed=seed)
    x = W.uniform(35, seed + 1)
    g = W.uniform(45, seed + 2)
    alpha = 1.5
    gx, gv, bound = oracle.backward(*A.astuple(), A.n_cols, g, x, alpha, with_bound=True)
    assert within(gx, alpha * dense_of(A).T @ g, bound, 1e-13)
    # f(val) = g^T (alpha A(val) x) is linear in val: central differences are exact
    h = 1e-3
    for k in range(A.nnz):
        vp = A.val.copy(); vp[k] += h
        vm = A.val.copy(); vm[k] -= h
        dy = oracle.spmv(A.row_ptr, A.col_idx, vp, x, alpha) - oracle.spmv(A.row_ptr, A.col_idx, vm, x, alpha)
        assert (g @ dy) / (2 * h) == pytest.approx(gv[k], rel=1e-9, abs=1e-12)
    # Euler identity for a form linear in val: sum_k val_k grad_val_k = g^T(alpha A x)
    f = g @ oracle.spmv(*A.astuple(), x, alpha)
    assert np.dot(A.val, gv) == pytest.approx(f, rel=1e-12, abs=1e-12)
    assert np.dot(gx, x) == pytest.approx(f, rel=1e-12, abs=1e-12)


def test_fd_on_27pt_16cubed():
    A = W.stencil27(W.STENCIL27_FD_GRID, seed=W.SEED_STENCIL27_VAL)
    x = W.uniform(A.n_cols, W.SEED_STENCIL27_X)
    g = W.uniform(A.n_rows, W.SEED_STENCIL27_G)
    gx, gv = oracle.backward(*A.astuple(), A.n_cols, g, x)
    rng = np.random.default_rng(0)
    h = 1e-3
    for k in rng.choice(A.nnz, 20, replace=False):
        vp = A.val.copy(); vp[k] += h
        vm = A.val.copy(); vm[k] -= h
        # difference the outputs before the reduction with g so the central
        # difference does not cancel against the size of f
        dy = oracle.spmv(A.row_ptr, A.col_idx, vp, x) - oracle.spmv(A.row_ptr, A.col_idx, vm, x)
        fd = (g @ dy) / (2 * h)
        assert fd == pytest.approx(gv[k], rel=1e-9, abs=1e-12)
    # grad_x by central differences in x (also linear)
    for j in rng.choice(A.n_cols, 10, replace=False):
        xp = x.copy(); xp[j] += h
        xm = x.copy(); xm[j] -= h
        dy = oracle.spmv(*A.astuple(), xp) - oracle.spmv(*A.astuple(), xm)
        fd = (g @ dy) / (2 * h)
        assert fd == pytest.approx(gx[j], rel=1e-9, abs=1e-12)


@pytest.mark.parametrize("nb", [1, 2, 3, 8])
@pytest.mark.parametrize("seed", [1, 5])
def test_split_blocks_definition(nb, seed):
    A = W.random_csr(97, 97, seed=seed, empty_frac=0.3)
    bs = oracle.split_blocks(A.row_ptr, nb)
    nnz = A.nnz
    ref = [0] + [int(np.searchsorted(A.row_ptr, -(-b * nnz // nb), side="left")) for b in range(1, nb)] + [A.n_rows]
    ref = [min(r, A.n_rows) for r in ref]
    assert list(bs) == ref
    assert np.all(np.diff(bs) >= 0)
    maxlen = int(np.diff(A.row_ptr).max())
    for b in range(nb):
        blk = A.row_ptr[bs[b + 1]] - A.row_ptr[bs[b]]
        assert abs(blk - nnz / nb) <= maxlen + 1


@pytest.mark.parametrize("nb", [1, 4, 8])
def test_split_halo_brute_force(nb):
    A = W.random_csr(120, 120, seed=nb, empty_frac=0.1)
    bs = oracle.split_blocks(A.row_ptr, nb)
    cnt, hmap, nl, nn = oracle.split_halo(A.row_ptr, A.col_idx, A.n_cols, bs)
    off = 0
    for b in range(nb):
        lo, hi = bs[b], bs[b + 1]
        cols = [int(c) for i in range(lo, hi) for c in A.col_idx[A.row_ptr[i]:A.row_ptr[i + 1]]]
        halo = sorted({c for c in cols if not (lo <= c < hi)})
        assert cnt[b] == len(halo)
        assert list(hmap[off:off + cnt[b]]) == halo
        assert nl[b] == sum(1 for c in cols if lo <= c < hi)
        assert nn[b] == sum(1 for c in cols if not (lo <= c < hi))
        off += cnt[b]
    assert off == hmap.size


def test_split_sum_equals_plain():
    """The local part plus the nonlocal part through the halo is the plain product
    (the split only regroups the row sum, Sect. 3.4)."""
    A = W.hamiltonian_like(2000, seed=11)
    x = W.uniform(2000, 3)
    bs = oracle.split_blocks(A.row_ptr, 8)
    cnt, hmap, _, _ = oracle.split_halo(A.row_ptr, A.col_idx, A.n_cols, bs)
    halo = x[hmap]
    rows = np.repeat(np.arange(A.n_rows), np.diff(A.row_ptr))
    blk = np.searchsorted(bs, rows, side="right") - 1
    local = (A.col_idx >= bs[blk]) & (A.col_idx < bs[blk + 1])
    starts = np.concatenate([[0], np.cumsum(cnt)])
    hcol = np.zeros(A.nnz, np.int64)
    for b in range(8):
        sel = (~local) & (blk == b)
        hcol[sel] = starts[b] + np.searchsorted(hmap[starts[b]:starts[b + 1]], A.col_idx[sel])
    assert np.array_equal(halo[hcol[~local]], x[A.col_idx[~local]])
    y = oracle.spmv(*A.astuple(), x)
    vl = np.where(local, A.val, 0.0)
    vn = np.where(local, 0.0, A.val)
    yl = oracle.spmv(A.row_ptr, A.col_idx, vl, x)
    yn = oracle.spmv(A.row_ptr, np.where(local, 0, hcol).astype(np.int32), vn, halo if halo.size else np.zeros(1))
    _, bound = oracle.spmv(*A.astuple(), x, with_bound=True)
    assert within(yl + yn, y, bound, 1e-13)


def test_cg_solves_spd():
    A = W.laplace2d(20)
    xs = W.uniform(A.n_rows, 1)
    b = oracle.spmv(*A.astuple(), xs)
    x, it = oracle.cg(*A.astuple(), b, tol=1e-12, maxit=2000)
    r = oracle.residual(*A.astuple(), b, x)
    assert np.linalg.norm(r) <= 1e-12 * np.linalg.norm(b) * 1.0001
    ref = np.linalg.solve(dense_of(A), b)
    lmax = 8 * math.cos(math.pi / 42) ** 2
    lmin = 8 * math.sin(math.pi / 42) ** 2
    assert np.linalg.norm(x - ref) <= (lmax / lmin) * 1e-12 * np.linalg.norm(ref) * 10
    assert 20 < it < 400


def test_row_histogram():
    A = W.random_csr(500, 100, seed=3, max_len=30, long_rows=3, long_len=90)
    h = oracle.row_histogram(A.row_ptr, 40)
    lens = np.diff(A.row_ptr)
    ref = np.bincount(np.minimum(lens, 39), minlength=40)
    assert np.array_equal(h, ref)


def expand_symmetric(U):
    """Full CRS of U + U_s^T (U_s: U without its diagonal), entries summed."""
    import scipy.sparse as sp
    n = U.n_rows
    M = sp.csr_matrix((U.val, U.col_idx, U.row_ptr), shape=(n, n))
    D = sp.diags(M.diagonal())
    F = (M + M.T - D).tocsr()
    F.sum_duplicates()
    F.sort_indices()
    return W.CRS(F.indptr.astype(np.int32), F.indices.astype(np.int32), F.data, n)


@pytest.mark.parametrize("n", [1, 2, 17, 64, 300])
@pytest.mark.parametrize("seed", [1, 2])
def test_spmv_sym_vs_dense_and_full(n, seed):
    U = W.random_symmetric_upper(n, seed)
    x = W.uniform(n, seed + 10)
    y0 = W.uniform(n, seed + 20)
    D = dense_of(U)
    full = D + np.triu(D, 1).T
    F = expand_symmetric(U)
    for alpha, beta in [(1.0, 0.0), (-0.5, 1.0), (2.0, -3.0), (0.0, 1.5)]:
        y, bound = oracle.spmv_sym(*U.astuple(), x, alpha, beta, y0, with_bound=True)
        ref = alpha * (full @ x) + (beta * y0 if beta != 0 else 0.0)
        assert within(y, ref, bound, 1e-13)
        yf, bf = oracle.spmv(*F.astuple(), x, alpha, beta, y0, with_bound=True)
        assert within(y, yf, bound, 1e-13)


def test_spmv_sym_integer_exact_and_laplacians():
    for A in (W.laplace2d(12), W.laplace3d(6), W.hamiltonian_like(3000, seed=7)):
        U = W.upper_triangle(A)
        x = W.integers(A.n_rows, 5).astype(np.float64)
        if A.n_rows == 3000:  # random values: tolerance; the stencils: exact
            y, bound = oracle.spmv_sym(*U.astuple(), x, with_bound=True)
            assert within(y, oracle.spmv(*A.astuple(), x), bound, 1e-13)
        else:
            assert np.array_equal(oracle.spmv_sym(*U.astuple(), x), oracle.spmv(*A.astuple(), x))
    Ui = W.random_symmetric_upper(200, 3, integer=True)
    xi = W.integers(200, 6).astype(np.float64)
    Fi = expand_symmetric(Ui)
    assert np.array_equal(oracle.spmv_sym(*Ui.astuple(), xi), oracle.spmv(*Fi.astuple(), xi))
