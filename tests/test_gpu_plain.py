"""GPU parity of the plain product y = alpha*A*x + beta*y (Listing 1) against the
oracle, through the C ABI: irregular small matrices under every kernel plan,
edge cases, and the full 2D 5-point (256^2) and 3D 7-point (160^3) operators."""
import numpy as np
import pytest

import oracle
from paper_1106_5908_gb300 import workloads as W
from gpu_util import assert_bitexact, assert_within, dev, host, need_gpu

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

PLANS = [(6, 7), (6, 9), (0, 15), (0, 7), (3, 7), (3, 15), (4, 7), (4, 9), (4, 11), (4, 15), (5, 32), (5, 256), (5, 4096),
         (0, 16), (0, 8), (2, 7), (2, 15), (2, 31), (1, 1), (1, 2), (1, 4), (1, 8), (1, 16), (1, 32)]
N_CHUNK_PLANS = 18  # plans before the row-vector kernel


def make(A, dtype=None):
    from paper_1106_5908_gb300 import Matrix
    return Matrix.from_csr(A.row_ptr, A.col_idx, A.val, A.n_cols, dtype=dtype)


@pytest.fixture(autouse=True)
def _gpu():
    need_gpu()


@pytest.mark.parametrize("shape", [(1, 1), (7, 5), (64, 64), (300, 200), (3000, 2500), (20000, 20000)])
@pytest.mark.parametrize("plan", PLANS)
def test_random_plans(shape, plan):
    A = W.random_csr(*shape, seed=shape[0] + plan[1], max_len=24)
    M = make(A)
    M.set_plan(*plan)
    x = W.uniform(A.n_cols, 3)
    y0 = W.uniform(A.n_rows, 4)
    for alpha, beta in [(1.0, 0.0), (-0.75, 1.0), (2.0, -0.5), (0.0, 2.0)]:
        ref, bound = oracle.spmv(*A.astuple(), x, alpha, beta, y0, with_bound=True)
        y = dev(y0)
        M.apply(dev(x), y, alpha, beta)
        assert_within(host(y), ref, bound, 1e-13, f"plan {plan} a={alpha} b={beta}")


@pytest.mark.parametrize("plan", PLANS[:N_CHUNK_PLANS])
@pytest.mark.parametrize("long_len", [253, 257, 509, 513, 1791, 1793, 3841, 9000, 40000])
def test_long_rows(plan, long_len):
    """Rows longer than a tile take the CTA-wide path; mixed with short ones."""
    A = W.random_csr(400, 5000, seed=long_len, max_len=30, long_rows=5, long_len=long_len)
    M = make(A)
    M.set_plan(*plan)
    x = W.uniform(A.n_cols, 5)
    ref, bound = oracle.spmv(*A.astuple(), x, with_bound=True)
    y = M.apply(dev(x))
    assert_within(host(y), ref, bound, 1e-13, f"long rows {long_len}")
    info = M.info()
    if plan[0] == 2:
        cap = {7: 1792, 15: 3840, 31: 7936}[plan[1]]
        assert info["long_rows"] == int((np.diff(A.row_ptr) > cap).sum())
    elif plan[0] == 4:
        # slot-major chunks start at the row's first entry
        assert info["long_rows"] == int((np.diff(A.row_ptr) > 32 * plan[1]).sum())
    elif plan[0] == 5:
        # rows of more than 128 entries leave the sorted slices
        assert info["long_rows"] == int((np.diff(A.row_ptr) > 128).sum())
    else:
        # a row is long when it does not fit 32*E slots from the aligned start
        slots = 32 * plan[1]
        lens = A.row_ptr[1:].astype(np.int64) - (A.row_ptr[:-1] & ~3)
        assert info["long_rows"] == int((lens > slots).sum())


@pytest.mark.parametrize("plan", PLANS)
def test_integer_bitexact(plan):
    A = W.random_csr(5000, 4000, seed=11, integer=True, max_len=40, long_rows=2, long_len=5000)
    M = make(A)
    M.set_plan(*plan)
    x = W.integers(A.n_cols, 12)
    y0 = W.integers(A.n_rows, 13)
    y = dev(y0)
    M.apply(dev(x), y, 1.0, 1.0)
    assert_bitexact(host(y), oracle.spmv(*A.astuple(), x, 1.0, 1.0, y0), f"integer {plan}")


def test_edge_cases():
    from paper_1106_5908_gb300 import Matrix
    # no rows
    M = Matrix.from_csr(np.zeros(1, np.int32), np.zeros(0, np.int32), np.zeros(0), 5)
    assert M.apply(dev(np.ones(5))).numel() == 0
    # rows but no entries: y = beta*y
    M = Matrix.from_csr(np.zeros(11, np.int32), np.zeros(0, np.int32), np.zeros(0), 4)
    y0 = W.uniform(10, 1)
    y = dev(y0)
    M.apply(dev(np.ones(4)), y, 2.0, 0.5)
    assert_bitexact(host(y), 0.5 * y0)
    # no columns
    M = Matrix.from_csr(np.zeros(4, np.int32), np.zeros(0, np.int32), np.zeros(0), 0)
    y = M.apply(torch.zeros(0, dtype=torch.float64, device="cuda"), dev(np.full(3, 7.0)), 1.0, 1.0)
    assert_bitexact(host(y), np.full(3, 7.0))
    # beta == 0 does not read y
    A = W.random_csr(500, 500, seed=2)
    M = make(A)
    x = W.uniform(500, 2)
    y = dev(np.full(500, np.nan))
    M.apply(dev(x), y, 1.5, 0.0)
    ref, bound = oracle.spmv(*A.astuple(), x, 1.5, 0.0, with_bound=True)
    assert np.all(np.isfinite(host(y)))
    assert_within(host(y), ref, bound, 1e-13)


def test_device_pointer_create_and_set_values():
    from paper_1106_5908_gb300 import Matrix
    A = W.random_csr(2000, 1500, seed=21)
    M = Matrix.from_csr(dev(A.row_ptr), dev(A.col_idx), dev(A.val), A.n_cols)
    x = W.uniform(A.n_cols, 1)
    ref, bound = oracle.spmv(*A.astuple(), x, with_bound=True)
    assert_within(host(M.apply(dev(x))), ref, bound, 1e-13)
    v2 = W.uniform(A.nnz, 9)
    M.set_values(dev(v2))
    ref2, bound2 = oracle.spmv(A.row_ptr, A.col_idx, v2, x, with_bound=True)
    assert_within(host(M.apply(dev(x))), ref2, bound2, 1e-13)


def test_histogram_matches_oracle():
    A = W.random_csr(3000, 100, seed=5, max_len=50, long_rows=4, long_len=300)
    M = make(A)
    assert np.array_equal(M.histogram(64), oracle.row_histogram(A.row_ptr, 64))


@pytest.mark.parametrize("plan", [(0, 16), (0, 8), (2, 15), (1, 4)])
def test_laplace2d_256(plan):
    A = W.laplace2d(W.LAPLACE2D_GRID)
    assert (A.n_rows, A.nnz) == (65536, 326656)
    M = make(A)
    M.set_plan(*plan)
    x = W.uniform(A.n_rows, W.SEED_LAPLACE2D_X)
    ref, bound = oracle.spmv(*A.astuple(), x, with_bound=True)
    assert_within(host(M.apply(dev(x))), ref, bound, 1e-13, "5-point 256^2 uniform")
    xi = W.integers(A.n_rows, W.SEED_LAPLACE2D_XINT)
    assert_bitexact(host(M.apply(dev(xi))), oracle.spmv(*A.astuple(), xi), "5-point 256^2 integer")


@pytest.fixture(scope="module")
def poisson7():
    return W.laplace3d(W.POISSON7_GRID)


def test_laplace3d_160(poisson7):
    A = poisson7
    assert (A.n_rows, A.nnz) == (4096000, 28518400)
    M = make(A)
    x = W.uniform(A.n_rows, W.SEED_POISSON7_B)
    ref, bound = oracle.spmv(*A.astuple(), x, with_bound=True)
    assert_within(host(M.apply(dev(x))), ref, bound, 1e-13, "7-point 160^3 FP64")
    xi = W.integers(A.n_rows, 7)
    assert_bitexact(host(M.apply(dev(xi))), oracle.spmv(*A.astuple(), xi), "7-point 160^3 integer")


@pytest.mark.parametrize("acc", ["ff", "f64"])
@pytest.mark.parametrize("ydt", ["f32", "f64"])
def test_fp32_storage_small(acc, ydt):
    A = W.random_csr(6000, 5000, seed=17, max_len=40, long_rows=3, long_len=4500)
    v32 = A.val.astype(np.float32)
    x32 = W.uniform(A.n_cols, 2).astype(np.float32)
    M = make(W.CRS(A.row_ptr, A.col_idx, v32, A.n_cols))
    M.set_accumulator(acc)
    yt = torch.float32 if ydt == "f32" else torch.float64
    y0 = W.uniform(A.n_rows, 3)
    ref, bound = oracle.spmv(A.row_ptr, A.col_idx, v32.astype(np.float64), x32.astype(np.float64),
                             0.5, 1.0, y0.astype(np.float32).astype(np.float64) if ydt == "f32" else y0,
                             with_bound=True)
    y = dev(y0.astype(np.float32) if ydt == "f32" else y0)
    M.apply(dev(x32), y, 0.5, 1.0)
    assert y.dtype == yt
    assert_within(host(y), ref, bound, 1e-6, f"fp32 storage acc={acc} y={ydt}")


def test_fp32_storage_integer_bitexact():
    A = W.random_csr(4000, 3000, seed=19, integer=True, max_len=30)
    M = make(W.CRS(A.row_ptr, A.col_idx, A.val.astype(np.float32), A.n_cols))
    x = W.integers(A.n_cols, 4).astype(np.float32)
    ref = oracle.spmv(*A.astuple(), x.astype(np.float64))
    assert_bitexact(host(M.apply(dev(x))).astype(np.float64), ref, "fp32 integer")
    assert_bitexact(host(M.apply(dev(x), out_dtype=torch.float64)), ref, "fp32->f64 integer")


def test_laplace3d_160_fp32(poisson7):
    A = poisson7
    M = make(W.CRS(A.row_ptr, A.col_idx, A.val.astype(np.float32), A.n_cols))
    x = W.uniform(A.n_rows, W.SEED_POISSON7_B).astype(np.float32)
    ref, bound = oracle.spmv(*A.astuple(), x.astype(np.float64), with_bound=True)
    assert_within(host(M.apply(dev(x))), ref, bound, 1e-6, "7-point 160^3 FP32")


def test_autotuner_choices():
    """The tuner picks the sorted row-slice kernel (windows of 4096 rows) for
    matrices whose columns stay near the previous row's (stencils): in FP64 with
    at least 12 entries per row, with FP32 storage at any row length; otherwise
    the chunk kernels: FP64 the slot-major one with 7 entries per lane for short
    rows and 9 otherwise, FP32 storage the slot-major one with 9.  A matrix whose
    sorted slices would pad more than 10 % keeps the chunk kernels."""
    from paper_1106_5908_gb300 import Matrix
    H = W.hamiltonian_like(50000, seed=3)
    L3 = W.laplace3d(24)
    S27 = W.stencil27(20, seed=1)
    for A, want in ((H, (4, 9)), (L3, (4, 7)), (S27, (5, 4096))):
        info = Matrix.from_csr(A.row_ptr, A.col_idx, A.val, A.n_cols).info()
        assert (info["family"], info["E"]) == want
    for A, want in ((H, (4, 9)), (L3, (5, 4096)), (S27, (5, 4096))):
        info = Matrix.from_csr(A.row_ptr, A.col_idx, A.val, A.n_cols, dtype=torch.float32).info()
        assert (info["family"], info["E"]) == want
    # 100 rows of lengths 100, 99, ..., 1 with columns 0 .. len-1 (not scattered,
    # 50.5 per row): one window, slices of widths 100 and 36 would store 8704
    # slots for 5050 entries, so the tuner keeps the slot-major chunk kernel
    n = 100
    lens = np.arange(n, 0, -1, dtype=np.int64)
    rp = np.zeros(n + 1, np.int32)
    rp[1:] = np.cumsum(lens)
    col = np.concatenate([np.arange(l, dtype=np.int32) for l in lens])
    info = Matrix.from_csr(rp, col, np.ones(rp[-1]), n).info()
    assert info["family"] == 4


@pytest.mark.parametrize("acc", ["ff", "f64"])
@pytest.mark.parametrize("plan", [(0, 7), (0, 15), (0, 16), (1, 1)])
def test_fp32_widening_exact(acc, plan):
    """FP32 inputs are widened to FP64 exactly, across every class of float: with
    a unit diagonal, y_i = x_i as a double (zeros, subnormals, the normal range
    ends, and for FP64 accumulation also infinities and NaN)."""
    rng = np.random.default_rng(5)
    bits = np.concatenate([
        np.array([0x00000000, 0x80000000, 0x00000001, 0x80000001, 0x007fffff, 0x807fffff, 0x00400000,
                  0x00800000, 0x80800000, 0x7f7fffff, 0xff7fffff, 0x3f800000, 0x33800000], np.uint32),
        rng.integers(1, 0x00800000, 64, dtype=np.uint32),                     # subnormals
        rng.integers(0x00800000, 0x7f800000, 256, dtype=np.uint32) | (rng.integers(0, 2, 256, dtype=np.uint32) << 31)])
    if acc == "f64":
        bits = np.concatenate([bits, np.array([0x7f800000, 0xff800000, 0x7fc00000, 0x7fa00001], np.uint32)])
    x32 = bits.view(np.float32)
    n = x32.size
    A = W.CRS(np.arange(n + 1, dtype=np.int32), np.arange(n, dtype=np.int32), np.ones(n, np.float32), n)
    M = make(A)
    M.set_accumulator(acc)
    M.set_plan(*plan)
    y = host(M.apply(dev(x32), out_dtype=torch.float64))
    want = x32.astype(np.float64)
    nan = np.isnan(want)
    assert np.array_equal(np.isnan(y), nan)
    assert np.array_equal(y[~nan], want[~nan]), np.flatnonzero(y[~nan] != want[~nan])[:8]


@pytest.mark.parametrize("plan", [(5, 32), (5, 256), (5, 4096), (4, 9), (6, 9), (6, 15)])
@pytest.mark.parametrize("shape", [(300, 200), (20000, 20000)])
def test_fp32_storage_plans(plan, shape):
    """FP32-stored values and vectors on the row-slice and slot-major kernels
    (float-float sums): random rows with empty and long ones, every alpha/beta
    form, against the oracle on the FP32 values at the FP32-storage bound."""
    A = W.random_csr(*shape, seed=shape[0] + plan[1], max_len=40, long_rows=3, long_len=min(shape[1], 3000))
    v32 = A.val.astype(np.float32)
    M = make(W.CRS(A.row_ptr, A.col_idx, v32, A.n_cols))
    M.set_plan(*plan)
    x32 = W.uniform(A.n_cols, 7).astype(np.float32)
    y32 = W.uniform(A.n_rows, 8).astype(np.float32)
    for alpha, beta in [(1.0, 0.0), (-0.75, 1.0), (2.0, -0.5), (1.0, 1.0)]:
        ref, bound = oracle.spmv(A.row_ptr, A.col_idx, v32.astype(np.float64), x32.astype(np.float64), alpha,
                                 beta, y32.astype(np.float64), with_bound=True)
        y = dev(y32)
        M.apply(dev(x32), y, alpha, beta)
        assert_within(host(y), ref, bound, 1e-6, f"fp32 {plan} a={alpha} b={beta}")


@pytest.mark.parametrize("plan", [(4, 7), (4, 15), (5, 32), (5, 4096), (6, 9)])
def test_slot_major_follows_new_values(plan):
    """The slot-major copies (plan families 4 and 5) are laid out again after new
    values, in FP64 and in FP32 storage."""
    A = W.random_csr(5000, 4000, seed=41, max_len=40, long_rows=2, long_len=3000)
    x = W.uniform(A.n_cols, 1)
    for dt in (None, torch.float32):
        M = make(A, dtype=dt)
        M.set_plan(*plan)
        M.apply(dev(x if dt is None else x.astype(np.float32)))
        v2 = W.uniform(A.nnz, 2)
        M.set_values(dev(v2) if dt is None else dev(v2.astype(np.float32)))
        if dt is None:
            ref, bound = oracle.spmv(A.row_ptr, A.col_idx, v2, x, with_bound=True)
            assert_within(host(M.apply(dev(x))), ref, bound, 1e-13, f"slot-major f64 {plan}")
        else:
            v32 = v2.astype(np.float32).astype(np.float64)
            x32 = x.astype(np.float32)
            ref, bound = oracle.spmv(A.row_ptr, A.col_idx, v32, x32.astype(np.float64), with_bound=True)
            assert_within(host(M.apply(dev(x32))), ref, bound, 1e-6, f"slot-major f32 {plan}")
