"""FP32 storage on the slot-major kernel with E = 7 and 9 (the default FP32
accumulator there): each lane's piece of a row, at most E products, is summed
by plain FP32 FMAs and the pieces are joined by two-sum.  Recursive summation
of k terms errs by at most gamma_k * sum |a_ij x_j| with gamma_k = k u / (1 - k u),
u = 2^-24, so an FP64 result must lie within gamma_E of the oracle's sum of the
exact products (plus an FP64 rounding), which is tighter than the 1e-6 FP32
storage tolerance; rows whose FP32 sum is zero, tiny or not finite are summed
again with FP64 products."""
import numpy as np
import pytest

import oracle
from paper_1106_5908_gb300 import workloads as W
from gpu_util import dev, host, need_gpu

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

U = 2.0 ** -24


def gamma(k):
    return k * U / (1 - k * U)


@pytest.fixture(autouse=True)
def _gpu():
    need_gpu()


def make32(A, E):
    from paper_1106_5908_gb300 import Matrix
    M = Matrix.from_csr(A.row_ptr, A.col_idx, A.val.astype(np.float32), A.n_cols)
    M.set_plan(4, E)
    return M


def wide(rng, n, lo, hi):
    mag = np.exp2(rng.uniform(lo, hi, n))
    return (mag * np.where(rng.random(n) < 0.5, -1.0, 1.0)).astype(np.float32)


@pytest.mark.parametrize("E", [7, 9, 11])
@pytest.mark.parametrize("spread", [0.0, 24.0])
def test_error_within_gamma_E(E, spread):
    """Values and x with magnitudes spread over 2^+-spread (cancellation inside
    every lane's run): every row within gamma_E * sum |a_ij x_j| (+ 2^-52 of it
    for the FP64 result's own roundings)."""
    A = W.hamiltonian_like(150000, seed=11)
    rng = np.random.default_rng(E * 100 + int(spread))
    v = wide(rng, A.nnz, -spread, spread) if spread else A.val.astype(np.float32)
    x = wide(rng, A.n_cols, -spread, spread) if spread else W.uniform(A.n_cols, 5).astype(np.float32)
    A32 = W.CRS(A.row_ptr, A.col_idx, v, A.n_cols)
    M = make32(A32, E)
    ref, bound = oracle.spmv(A.row_ptr, A.col_idx, v.astype(np.float64), x.astype(np.float64), with_bound=True)
    y = host(M.apply(dev(x), out_dtype=torch.float64))
    err = np.abs(y - ref)
    lim = (gamma(E) + 2.0 ** -50) * bound
    bad = np.flatnonzero(~(err <= lim))
    assert bad.size == 0, (bad[:5], err[bad[:5]] / bound[bad[:5]])
    # and an FP32 result: the same, plus its rounding to float
    y32 = host(M.apply(dev(x))).astype(np.float64)
    lim32 = lim + U * (np.abs(ref) + gamma(E) * bound) * 1.0001
    bad = np.flatnonzero(~(np.abs(y32 - ref) <= lim32))
    assert bad.size == 0, bad[:5]


@pytest.mark.parametrize("E", [7, 9, 11])
def test_rows_summing_to_zero_are_exact(E):
    """A 2D Laplacian times a constant vector: interior rows sum to exactly 0 (a
    zero FP32 sum is re-summed in FP64), boundary rows to small integers: the
    result equals the oracle bit for bit, also with alpha/beta."""
    A = W.laplace2d(200)
    M = make32(A, E)
    x = np.full(A.n_cols, 3.0, np.float32)
    ref = oracle.spmv(*A.astuple(), x.astype(np.float64))
    assert np.count_nonzero(ref == 0.0) > A.n_rows // 2
    y = host(M.apply(dev(x), out_dtype=torch.float64))
    assert np.array_equal(y, ref)
    y0 = W.integers(A.n_rows, 3).astype(np.float64)
    ref2 = oracle.spmv(*A.astuple(), x.astype(np.float64), -2.0, 0.5, y0)
    yd = dev(y0)
    M.apply(dev(x), yd, -2.0, 0.5)
    assert np.array_equal(host(yd), ref2)


@pytest.mark.parametrize("E", [7, 9, 11])
def test_integer_values_bit_exact(E):
    """Integer values and x with every partial sum below 2^24: exact in FP32 runs
    and in the float-float joins, so bit-exact against the oracle."""
    A = W.hamiltonian_like(60000, seed=4)
    Ai = W.CRS(A.row_ptr, A.col_idx, np.rint(A.val * 3).astype(np.float32), A.n_cols)
    M = make32(Ai, E)
    x = W.integers(A.n_cols, 9).astype(np.float32)
    ref = oracle.spmv(Ai.row_ptr, Ai.col_idx, Ai.val.astype(np.float64), x.astype(np.float64))
    assert np.array_equal(host(M.apply(dev(x), out_dtype=torch.float64)), ref)
    assert np.array_equal(host(M.apply(dev(x))).astype(np.float64), ref)


def test_long_rows_use_float_float():
    """A row longer than a chunk (summed by a whole warp, lanes striding it) and
    chunks with empty rows (one row per lane) are not cut into runs of at most 9
    entries: they take the float-float sum (error of order (n u)^2 for a lane's
    n terms), far below gamma_9 even with wide magnitudes."""
    rng = np.random.default_rng(8)
    n = 2000
    lens = rng.integers(1, 12, n)
    lens[rng.random(n) < 0.05] = 0
    lens[17] = 5000
    lens[1200] = 900
    rp = np.zeros(n + 1, np.int64)
    rp[1:] = np.cumsum(lens)
    col = rng.integers(0, n, int(rp[-1])).astype(np.int32)
    v = wide(rng, int(rp[-1]), -12.0, 12.0)
    A = W.CRS(rp.astype(np.int32), col, v, n)
    x = wide(rng, n, -12.0, 12.0)
    for E in (7, 9, 11):
        M = make32(A, E)
        ref, bound = oracle.spmv(A.row_ptr, A.col_idx, v.astype(np.float64), x.astype(np.float64), with_bound=True)
        y = host(M.apply(dev(x), out_dtype=torch.float64))
        err = np.abs(y - ref)
        assert np.all(err <= (gamma(E) + 2.0 ** -50) * bound)
        for r in (17, 1200):
            assert err[r] <= 1e-9 * bound[r], (r, err[r] / bound[r])


# The row-slice kernel (family 5) takes FP32 runs when no row has more than 9
# entries: a lane's chain then covers a whole row.

def make_plan(A, plan):
    from paper_1106_5908_gb300 import Matrix
    M = Matrix.from_csr(A.row_ptr, A.col_idx, A.val.astype(np.float32), A.n_cols)
    M.set_plan(*plan)
    return M


@pytest.mark.parametrize("sigma", [32, 4096])
def test_row_slices_short_rows_within_gamma_7(sigma):
    A = W.laplace3d(40)
    rng = np.random.default_rng(sigma)
    v = wide(rng, A.nnz, -20.0, 20.0)
    x = wide(rng, A.n_cols, -20.0, 20.0)
    A32 = W.CRS(A.row_ptr, A.col_idx, v, A.n_cols)
    M = make_plan(A32, (5, sigma))
    ref, bound = oracle.spmv(A.row_ptr, A.col_idx, v.astype(np.float64), x.astype(np.float64), with_bound=True)
    y = host(M.apply(dev(x), out_dtype=torch.float64))
    assert np.all(np.abs(y - ref) <= (gamma(7) + 2.0 ** -50) * bound)
    y32 = host(M.apply(dev(x))).astype(np.float64)
    assert np.all(np.abs(y32 - ref) <= (gamma(7) + 2.0 ** -50) * bound + U * (np.abs(ref) + gamma(7) * bound) * 1.0001)


def test_row_slices_short_rows_exact_cases():
    """Rows that cancel to zero (a 3D Laplacian times a constant) and integer
    data: bit-exact on the row slices with FP32 runs."""
    A = W.laplace3d(30)
    M = make_plan(A, (5, 4096))
    x = np.full(A.n_cols, -2.0, np.float32)
    ref = oracle.spmv(*A.astuple(), x.astype(np.float64))
    assert np.count_nonzero(ref == 0.0) > A.n_rows // 2
    assert np.array_equal(host(M.apply(dev(x), out_dtype=torch.float64)), ref)
    xi = W.integers(A.n_cols, 6).astype(np.float32)
    ref = oracle.spmv(*A.astuple(), xi.astype(np.float64))
    assert np.array_equal(host(M.apply(dev(xi))).astype(np.float64), ref)


@pytest.mark.parametrize("plan", [(5, 256), (5, 4096), (4, 7), (4, 9)])
def test_short_rows_out_of_fp32_range(plan):
    """Values and x over FP32's whole exponent range on a 7-point pattern:
    products above FLT_MAX, below the subnormals and cancelling; every row within
    the FP32-storage bound of the oracle (rows the FP32 runs cannot guarantee are
    summed again in FP64), for FP32 and FP64 results and alpha/beta forms."""
    from test_gpu_fp32_range import check
    A = W.laplace3d(20)
    rng = np.random.default_rng(plan[1])
    v = wide(rng, A.nnz, -149.0, 127.0)
    x = wide(rng, A.n_cols, -149.0, 127.0)
    A32 = W.CRS(A.row_ptr, A.col_idx, v, A.n_cols)
    M = make_plan(A32, plan)
    y0 = W.uniform(A.n_rows, 4).astype(np.float32)
    for out in (torch.float32, torch.float64):
        out32 = out == torch.float32
        for alpha, beta in ((1.0, 0.0), (-0.5, 2.0)):
            yin = y0 if out32 else y0.astype(np.float64)
            ref, bound = oracle.spmv(A.row_ptr, A.col_idx, v.astype(np.float64), x.astype(np.float64), alpha, beta,
                                     yin.astype(np.float64), with_bound=True)
            y = dev(yin)
            M.apply(dev(x), y, alpha, beta)
            check(host(y), ref, bound, out32, f"plan {plan} out {out} a={alpha} b={beta}")


@pytest.mark.parametrize("sigma", [256, 4096])
def test_row_slices_long_rows_within_gamma_4(sigma):
    """27-point rows (up to 27 entries) on the row slices: FP32 runs of one block
    (4 slot rows) folded into float-float, so every row within gamma_4 of the
    oracle for any row length; and the reverse pass's row-slice copy of A^T."""
    A = W.stencil27(14, seed=2)
    rng = np.random.default_rng(sigma + 1)
    v = wide(rng, A.nnz, -20.0, 20.0)
    x = wide(rng, A.n_cols, -20.0, 20.0)
    A32 = W.CRS(A.row_ptr, A.col_idx, v, A.n_cols)
    M = make_plan(A32, (5, sigma))
    ref, bound = oracle.spmv(A.row_ptr, A.col_idx, v.astype(np.float64), x.astype(np.float64), with_bound=True)
    y = host(M.apply(dev(x), out_dtype=torch.float64))
    assert np.all(np.abs(y - ref) <= (gamma(4) + 2.0 ** -50) * bound)
    g = wide(rng, A.n_rows, -20.0, 20.0)
    gx_ref, _, gb = oracle.backward(A.row_ptr, A.col_idx, v.astype(np.float64), A.n_cols, g.astype(np.float64),
                                    x.astype(np.float64), 1.0, with_bound=True)
    for rep in range(2):
        gx, _ = M.backward(dev(g), dev(x))
        err = np.abs(host(gx).astype(np.float64) - gx_ref)
        assert np.all(err <= (gamma(9) + 2.0 ** -50) * gb + U * (np.abs(gx_ref) + gamma(9) * gb) * 1.0001), rep


def test_ir_cg_on_both_inner_paths():
    """IR-CG takes q = A p with p.q reduced by the row-slice product itself when its
    FP32 copy runs on the row slices (7-point matrix), and the product followed by
    a separate dot otherwise (a scattered, diagonally dominant symmetric matrix on
    the slot-major kernel): both converge to ||b - Ax|| <= 1e-12 ||b||, checked
    by the oracle."""
    from paper_1106_5908_gb300 import Matrix, ir_cg
    H = W.hamiltonian_like(60000, seed=21)
    rows = np.repeat(np.arange(H.n_rows), np.diff(H.row_ptr.astype(np.int64)))
    off = rows != H.col_idx
    v = H.val.copy()
    rowabs = np.bincount(rows[off], weights=np.abs(v[off]), minlength=H.n_rows)
    v[~off] = rowabs[rows[~off]] + 1.0  # diagonally dominant: SPD
    S = W.CRS(H.row_ptr, H.col_idx, v, H.n_cols)
    for A in (W.laplace3d(30), S):
        M = Matrix.from_csr(A.row_ptr, A.col_idx, A.val, A.n_cols)
        b = W.uniform(A.n_rows, 31)
        x, st = ir_cg(M, dev(b), outer_tol=1e-12, max_outer=50)
        assert st["converged"], st
        r = oracle.residual(A.row_ptr, A.col_idx, A.val, b, host(x))
        assert np.linalg.norm(r) / np.linalg.norm(b) <= 1.5e-12, st
