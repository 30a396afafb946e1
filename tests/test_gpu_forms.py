"""GPU parity of the extended forms: block vectors, the reverse pass (transposed
structure bit-exact; gradients against the oracle, central differences and torch
autograd), the CG solvers, and the batched persistent launch."""
import numpy as np
import pytest

import oracle
from paper_1106_5908_gb300 import workloads as W
from gpu_util import assert_bitexact, assert_within, dev, host, need_gpu

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(autouse=True)
def _gpu():
    need_gpu()


def make(A):
    from paper_1106_5908_gb300 import Matrix
    return Matrix.from_csr(A.row_ptr, A.col_idx, A.val, A.n_cols)


# ---------------------------------------------------------------- block vectors

@pytest.mark.parametrize("nrhs", [1, 2, 3, 4, 5, 8, 16, 31, 32, 33, 64])
def test_spmm_small(nrhs):
    A = W.random_csr(3000, 2000, seed=nrhs, max_len=40, long_rows=2, long_len=2500)
    M = make(A)
    X = W.uniform(0, 1, shape=(A.n_cols, nrhs))
    Y0 = W.uniform(0, 2, shape=(A.n_rows, nrhs))
    for alpha, beta in [(1.0, 0.0), (0.5, -1.5)]:
        ref, bound = oracle.spmm(*A.astuple(), X, alpha, beta, Y0, with_bound=True)
        Y = dev(Y0)
        M.spmm(dev(X), Y, alpha, beta)
        assert_within(host(Y).ravel(), ref.ravel(), bound.ravel(), 1e-13, f"nrhs={nrhs}")


@pytest.mark.parametrize("nrhs", [4, 6, 7, 8])
def test_spmm_stencil_and_padded(nrhs):
    """Block vectors on the sorted row slices of a 27-point stencil (groups of 4
    right-hand sides there, the rest on the tile kernel), and on a matrix whose
    slices would pad too much (rows of lengths 200, 199, ..., 1 plus a long one:
    the tile kernel alone)."""
    S = W.stencil27(12, seed=nrhs)
    n = 200
    lens = np.arange(n, 0, -1, dtype=np.int64)
    rp = np.zeros(n + 1, np.int32)
    rp[1:] = np.cumsum(lens)
    rng = np.random.default_rng(nrhs)
    col = np.concatenate([np.sort(rng.choice(300, int(l), replace=False)).astype(np.int32) for l in lens])
    P = W.CRS(rp, col, rng.uniform(-1, 1, rp[-1]), 300)
    for A in (S, P):
        M = make(A)
        X = W.uniform(0, 5, shape=(A.n_cols, nrhs))
        Y0 = W.uniform(0, 6, shape=(A.n_rows, nrhs))
        for alpha, beta in [(1.0, 0.0), (-2.0, 0.5)]:
            ref, bound = oracle.spmm(*A.astuple(), X, alpha, beta, Y0, with_bound=True)
            Y = dev(Y0)
            M.spmm(dev(X), Y, alpha, beta)
            assert_within(host(Y).ravel(), ref.ravel(), bound.ravel(), 1e-13, f"nrhs={nrhs} n={A.n_rows}")


def test_spmm_integer_bitexact():
    A = W.random_csr(2000, 2000, seed=3, integer=True, max_len=30)
    M = make(A)
    X = np.random.default_rng(1).integers(-8, 9, (2000, 8)).astype(np.float64)
    assert_bitexact(host(M.spmm(dev(X))).ravel(), oracle.spmm(*A.astuple(), X).ravel())


# ---------------------------------------------------------------- reverse pass

@pytest.mark.parametrize("shape", [(1, 1), (50, 40), (700, 900), (4000, 3000)])
def test_transpose_structure_bitexact(shape):
    A = W.random_csr(*shape, seed=shape[0], max_len=30, long_rows=1, long_len=min(shape[1], 5000))
    M = make(A)
    rpt, cit, perm = M.transpose_structure()
    ort, oct_, operm = oracle.transpose(A.row_ptr, A.col_idx, A.n_cols)
    assert_bitexact(rpt, ort, "rowT_ptr")
    assert_bitexact(cit, oct_, "colT")
    assert_bitexact(perm, operm, "perm")


@pytest.mark.parametrize("case", ["dense_column", "medium_columns", "all_one_column"])
def test_transpose_long_columns(case):
    """Long columns of A (long rows of A^T): one column with an entry in each of
    100,000 rows, or 200 columns of about 3000 entries, or every entry in one
    column; the structure is bit-exact against the oracle (the column order is a
    stable radix sort, linear in the entries), and grad_x = A^T g on it is
    within the bound (first pass through the permutation, second on the
    laid-out copy)."""
    import time
    if case == "dense_column":
        A = W.column_heavy_csr(100000, 50000, seed=5, dense=1, medium=0)
    elif case == "medium_columns":
        A = W.column_heavy_csr(60000, 40000, seed=6, dense=0, medium=200, medium_len=3000)
    else:
        n = 70000
        A = W.CRS(np.arange(n + 1, dtype=np.int32), np.full(n, 123, np.int32), W.uniform(n, 7), 500)
    M = make(A)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    rpt, cit, perm = M.transpose_structure()
    build_s = time.perf_counter() - t0
    ort, oct_, operm = oracle.transpose(A.row_ptr, A.col_idx, A.n_cols)
    assert_bitexact(rpt, ort, "rowT_ptr")
    assert_bitexact(cit, oct_, "colT")
    assert_bitexact(perm, operm, "perm")
    assert build_s < 5.0, build_s
    x = W.uniform(A.n_cols, 8)
    g = W.uniform(A.n_rows, 9)
    rgx, rgv, bound = oracle.backward(*A.astuple(), A.n_cols, g, x, with_bound=True)
    for _ in range(2):
        gx, gv = M.backward(dev(g), dev(x))
        assert_within(host(gx), rgx, bound, 1e-13, f"grad_x {case}")
        assert_bitexact(host(gv), rgv, f"grad_val {case}")


@pytest.mark.parametrize("alpha", [1.0, -0.5])
def test_backward_small(alpha):
    A = W.random_csr(3000, 2500, seed=9, max_len=30, long_rows=2, long_len=4500)
    M = make(A)
    x = W.uniform(A.n_cols, 1)
    g = W.uniform(A.n_rows, 2)
    gx, gv = M.backward(dev(g), dev(x), alpha)
    rgx, rgv, bound = oracle.backward(*A.astuple(), A.n_cols, g, x, alpha, with_bound=True)
    assert_within(host(gx), rgx, bound, 1e-13, "grad_x")
    if alpha == 1.0:
        assert_bitexact(host(gv), rgv, "grad_val")
    else:
        assert_within(host(gv), rgv, np.abs(rgv), 2.5e-16, "grad_val")


@pytest.mark.parametrize("kind", ["random", "stencil27"])
def test_backward_after_new_values(kind):
    """The transposed values are rebuilt after spmv_set_values, and an autograd
    graph whose forward ran before another one still uses its own values (A^T on
    the slot-major copy for scattered columns, on the row slices for a stencil)."""
    from paper_1106_5908_gb300 import spmv
    A = W.random_csr(2000, 1800, seed=21, max_len=25) if kind == "random" else W.stencil27(13, seed=21)
    M = make(A)
    x = W.uniform(A.n_cols, 3)
    g = W.uniform(A.n_rows, 4)
    M.backward(dev(g), dev(x))
    v2 = W.uniform(A.nnz, 5)
    M.set_values(dev(v2))
    for _ in range(2):  # rebuilt once, then reused
        gx, _ = M.backward(dev(g), dev(x), need_val=False)
        rgx, _, bound = oracle.backward(A.row_ptr, A.col_idx, v2, A.n_cols, g, x, with_bound=True)
        assert_within(host(gx), rgx, bound, 1e-13, "grad_x after set_values")
    val1 = dev(A.val).requires_grad_(False)
    val2 = dev(v2).requires_grad_(False)
    xa = dev(x).requires_grad_(True)
    xb = dev(x).requires_grad_(True)
    y1 = spmv(M, val1, xa)
    y2 = spmv(M, val2, xb)
    y1.backward(dev(g))
    y2.backward(dev(g))
    r1, _, b1 = oracle.backward(*A.astuple(), A.n_cols, g, x, with_bound=True)
    r2, _, b2 = oracle.backward(A.row_ptr, A.col_idx, v2, A.n_cols, g, x, with_bound=True)
    assert_within(host(xa.grad), r1, b1, 1e-13, "first graph")
    assert_within(host(xb.grad), r2, b2, 1e-13, "second graph")


@pytest.fixture(scope="module")
def st27():
    return W.stencil27(W.STENCIL27_GRID, seed=W.SEED_STENCIL27_VAL)


@pytest.mark.parametrize("nrhs", [4, 8, 16, 32])
def test_block_vectors_27pt_128(st27, nrhs):
    """Block vectors on the full 128^3 27-point matrix (row slices, groups of 4),
    every row of Y against the oracle."""
    A = st27
    M = make(A)
    X = W.uniform(0, W.SEED_BLOCK_X + nrhs, shape=(A.n_cols, nrhs))
    ref, bound = oracle.spmm(*A.astuple(), X, with_bound=True)
    assert_within(host(M.spmm(dev(X))).ravel(), ref.ravel(), bound.ravel(), 1e-13, f"27-point nrhs={nrhs}")


def test_backward_27pt_128(st27):
    A = st27
    assert (A.n_rows, A.nnz) == (2097152, 55742968)
    M = make(A)
    x = W.uniform(A.n_cols, W.SEED_STENCIL27_X)
    g = W.uniform(A.n_rows, W.SEED_STENCIL27_G)
    ref, bound = oracle.spmv(*A.astuple(), x, with_bound=True)
    assert_within(host(M.apply(dev(x))), ref, bound, 1e-13, "27-point forward")
    rgx, rgv, gbound = oracle.backward(*A.astuple(), A.n_cols, g, x, with_bound=True)
    # the first reverse pass reads A^T's values through the permutation; the
    # second lays them out once and runs the row-slice kernel on A^T
    for rep in range(2):
        gx, gv = M.backward(dev(g), dev(x))
        assert_within(host(gx), rgx, gbound, 1e-13, f"27-point grad_x pass {rep}")
        assert_bitexact(host(gv), rgv, f"27-point grad_val pass {rep}")


def test_backward_27pt_fp32(st27):
    from paper_1106_5908_gb300 import Matrix
    A = st27
    v32 = A.val.astype(np.float32)
    M = Matrix.from_csr(A.row_ptr, A.col_idx, v32, A.n_cols)
    x = W.uniform(A.n_cols, W.SEED_STENCIL27_X).astype(np.float32)
    g = W.uniform(A.n_rows, W.SEED_STENCIL27_G).astype(np.float32)
    # the forward product on the autotuned plan (row slices, float-float sums)
    assert M.info()["family"] == 5
    ref, bound = oracle.spmv(A.row_ptr, A.col_idx, v32.astype(np.float64), x.astype(np.float64), with_bound=True)
    assert_within(host(M.apply(dev(x))), ref, bound, 1e-6, "27-point fp32 forward")
    rgx, rgv, gbound = oracle.backward(A.row_ptr, A.col_idx, v32.astype(np.float64), A.n_cols,
                                       g.astype(np.float64), x.astype(np.float64), with_bound=True)
    for rep in range(2):
        gx, gv = M.backward(dev(g), dev(x))
        assert_within(host(gx), rgx, gbound, 1e-6, f"27-point fp32 grad_x pass {rep}")
        assert_within(host(gv), rgv, np.abs(rgv), 1e-6, f"27-point fp32 grad_val pass {rep}")


def test_fd_16cubed_fp32_storage():
    """The FP32-storage reverse pass on the 16^3 27-point instance against central
    differences of f = g^T A(val) x computed by the library's own FP32-storage
    forward product (FP64 result): f is linear in each value and each x entry, so
    the quotient over the perturbation actually stored in FP32 is exact up to the
    forward product's rounding.  The forward runs with the FP64-FMA accumulator
    (exact products summed in FP64, the definition of the FP32-storage form): the
    quotient divides the forward's rounding by 2h = 0.02, and the default FP32-pipe
    accumulator's bound (a few 1e-7 of sum |a x| per row) would dominate it.  Also
    against the oracle's reverse pass."""
    A = W.stencil27(W.STENCIL27_FD_GRID, seed=W.SEED_STENCIL27_VAL)
    v32 = A.val.astype(np.float32)
    x32 = W.uniform(A.n_cols, W.SEED_STENCIL27_X).astype(np.float32)
    g32 = W.uniform(A.n_rows, W.SEED_STENCIL27_G).astype(np.float32)
    from paper_1106_5908_gb300 import Matrix
    M = Matrix.from_csr(A.row_ptr, A.col_idx, v32, A.n_cols)
    M.set_accumulator("f64")
    gd = dev(g32).double()
    for alpha in (1.0, 1.25):
        M.set_values(dev(v32))
        gx, gv = M.backward(dev(g32), dev(x32), alpha)
        gx, gv = host(gx).astype(np.float64), host(gv).astype(np.float64)
        rgx, rgv, gb = oracle.backward(A.row_ptr, A.col_idx, v32.astype(np.float64), A.n_cols,
                                       g32.astype(np.float64), x32.astype(np.float64), alpha, with_bound=True)
        assert_within(gx, rgx, gb, 1e-6, "fp32 grad_x vs oracle")
        assert_within(gv, rgv, np.abs(rgv), 1e-6, "fp32 grad_val vs oracle")

        def f(vals, xx):
            M.set_values(dev(vals))
            return alpha * torch.dot(gd, M.apply(dev(xx), out_dtype=torch.float64)).item()

        rng = np.random.default_rng(1)
        h = np.float32(1e-2)
        for k in rng.choice(A.nnz, 12, replace=False):
            vp = v32.copy(); vp[k] = v32[k] + h
            vm = v32.copy(); vm[k] = v32[k] - h
            fd = (f(vp, x32) - f(vm, x32)) / (float(vp[k]) - float(vm[k]))
            assert fd == pytest.approx(gv[k], rel=1e-6, abs=1e-9), ("val", k)
        for j in rng.choice(A.n_cols, 12, replace=False):
            xp = x32.copy(); xp[j] = x32[j] + h
            xm = x32.copy(); xm[j] = x32[j] - h
            fd = (f(v32, xp) - f(v32, xm)) / (float(xp[j]) - float(xm[j]))
            assert fd == pytest.approx(gx[j], rel=1e-6, abs=1e-6 * gb[j] + 1e-9), ("x", j)


def test_autograd_fd_16cubed():
    """SpMVFunction against central differences (torch.autograd.gradcheck) and
    against the oracle's reverse pass on the 16^3 27-point instance."""
    from paper_1106_5908_gb300 import spmv
    A = W.stencil27(W.STENCIL27_FD_GRID, seed=W.SEED_STENCIL27_VAL)
    M = make(A)
    val = dev(A.val).requires_grad_(True)
    x = dev(W.uniform(A.n_cols, W.SEED_STENCIL27_X)).requires_grad_(True)
    g = W.uniform(A.n_rows, W.SEED_STENCIL27_G)
    y = spmv(M, val, x, 1.25)
    y.backward(dev(g))
    rgx, rgv = oracle.backward(*A.astuple(), A.n_cols, g, host(x), 1.25)
    np.testing.assert_allclose(host(x.grad), rgx, rtol=1e-12, atol=1e-13)
    np.testing.assert_allclose(host(val.grad), rgv, rtol=1e-14, atol=0)
    # central differences on a few entries of val and x (f linear: exact to rounding)
    h = 1e-3
    gd = dev(g)
    rng = np.random.default_rng(0)
    with torch.no_grad():
        for k in rng.choice(A.nnz, 8, replace=False):
            vp = val.detach().clone(); vp[k] += h
            vm = val.detach().clone(); vm[k] -= h
            fd = (torch.dot(gd, spmv(M, vp, x.detach(), 1.25) - spmv(M, vm, x.detach(), 1.25)) / (2 * h)).item()
            assert fd == pytest.approx(float(host(val.grad)[k]), rel=1e-9, abs=1e-12)
    small = W.stencil27(4, seed=1)
    Ms = make(small)
    vs = dev(small.val).requires_grad_(True)
    xs = dev(W.uniform(small.n_cols, 2)).requires_grad_(True)
    assert torch.autograd.gradcheck(lambda v, xx: spmv(Ms, v, xx, 0.75), (vs, xs), eps=1e-6, atol=1e-8)


# ---------------------------------------------------------------- solvers

@pytest.mark.parametrize("grid", [24, W.POISSON7_GRID])
@pytest.mark.parametrize("inner", [(1e-3, 500), (1e-4, 200)])
def test_ir_cg_and_cg(grid, inner):
    from paper_1106_5908_gb300 import cg, ir_cg
    A = W.laplace3d(grid)
    M = make(A)
    b = W.uniform(A.n_rows, W.SEED_POISSON7_B)
    bd = dev(b)
    x, st = ir_cg(M, bd, outer_tol=1e-12, max_outer=50, inner_tol=inner[0], max_inner=inner[1])
    assert st["converged"], st
    xh = host(x)
    r = oracle.residual(*A.astuple(), b, xh)
    relres = np.linalg.norm(r) / np.linalg.norm(b)
    assert relres <= 1e-12 * 1.5, (relres, st)
    x64, st64 = cg(M, bd, tol=1e-12, max_iter=20000)
    assert st64["converged"], st64
    x64h = host(x64)
    r64 = oracle.residual(*A.astuple(), b, x64h)
    assert np.linalg.norm(r64) / np.linalg.norm(b) <= 1e-11, st64
    lam_max = 3 * (2 + 2 * np.cos(np.pi / (grid + 1)))
    lam_min = 3 * (2 - 2 * np.cos(np.pi / (grid + 1)))
    cond = lam_max / lam_min
    assert np.linalg.norm(xh - x64h) <= 2 * cond * 1e-11 * np.linalg.norm(x64h)


def test_ir_cg_manufactured_solution():
    from paper_1106_5908_gb300 import ir_cg
    A = W.laplace2d(64)
    M = make(A)
    xs = W.uniform(A.n_rows, 123)
    b = oracle.spmv(*A.astuple(), xs)
    x, st = ir_cg(M, dev(b), outer_tol=1e-12)
    assert st["converged"]
    n = 64
    cond = (2 + 2 * np.cos(np.pi / (n + 1))) / (2 - 2 * np.cos(np.pi / (n + 1)))
    assert np.linalg.norm(host(x) - xs) <= cond * 1e-12 * np.linalg.norm(xs) * 2


# ---------------------------------------------------------------- batched

@pytest.mark.parametrize("dtype", ["f64", "f32"])
def test_batched_small(dtype):
    from paper_1106_5908_gb300 import Batch, Matrix
    sizes = W.batch_sizes(24, seed=7, lo=50, hi=20000)
    srcs = [W.batch_matrix(m, int(n), seed=7) for m, n in enumerate(sizes)]
    # members with very short rows (about 2 entries per row) between them
    srcs[3:3] = [W.random_csr(n, n, seed=n, max_len=4, empty_frac=0.05) for n in (700, 5000, 20000)]
    mats, As = [], []
    for A in srcs:
        v = A.val.astype(np.float32) if dtype == "f32" else A.val
        As.append(W.CRS(A.row_ptr, A.col_idx, v, A.n_cols))
        mats.append(Matrix.from_csr(A.row_ptr, A.col_idx, v, A.n_cols))
    B = Batch(mats)
    # each member tuned from its own row lengths: 7 entries per lane below a
    # mean of 4 per row (the short-row members), else 9 (the Laplacians and the
    # Hamiltonian-like ones); both groups run in the one launch
    want_E = [7 if A.nnz / max(A.n_rows, 1) < 4 else 9 for A in As]
    info = B.info()
    assert info["member_E"] == want_E and len(set(want_E)) == 2
    assert info["E"] == 0
    tdt = torch.float32 if dtype == "f32" else torch.float64
    rel = 1e-6 if dtype == "f32" else 1e-13
    for rep, (alpha, beta) in enumerate([(1.0, 0.0), (1.0, 0.0), (-1.5, 0.5)]):
        xs = [W.uniform(A.n_cols, 100 + 7 * rep + m).astype(np.float32 if dtype == "f32" else np.float64)
              for m, A in enumerate(As)]
        y0s = [W.uniform(A.n_rows, 300 + m).astype(np.float32 if dtype == "f32" else np.float64)
               for m, A in enumerate(As)]
        xd = [dev(x) for x in xs]
        yd = [dev(y) for y in y0s]
        B.apply(xd, yd, alpha, beta)
        torch.cuda.synchronize()
        for m, A in enumerate(As):
            ref, bound = oracle.spmv(A.row_ptr, A.col_idx, A.val.astype(np.float64),
                                     xs[m].astype(np.float64), alpha, beta,
                                     y0s[m].astype(np.float64), with_bound=True)
            assert yd[m].dtype == tdt
            assert_within(host(yd[m]), ref, bound, rel, f"batch m={m} rep={rep}")


@pytest.mark.parametrize("dtype", ["f64", "f32"])
def test_batched_256_full_size(dtype):
    """The benchmark's batch at full size: 256 matrices, N ~ U[1000, 200000]
    (5-point Laplacians and Hamiltonian-like patterns, 235 M entries), FP64 and
    FP32 storage, one persistent launch replayed from a CUDA graph; every result
    against the oracle, for two right-hand sides (the second replay reuses the
    graph)."""
    from paper_1106_5908_gb300 import Batch, Matrix
    npdt = np.float32 if dtype == "f32" else np.float64
    tdt = torch.float32 if dtype == "f32" else torch.float64
    rel = 1e-6 if dtype == "f32" else 1e-13
    sizes = W.batch_sizes(W.BATCH_COUNT)
    As, mats = [], []
    for m, n in enumerate(sizes):
        A = W.batch_matrix(m, int(n))
        As.append(A)
        mats.append(Matrix.from_csr(A.row_ptr, A.col_idx, A.val.astype(npdt), A.n_cols))
    assert len(As) == 256 and sum(A.nnz for A in As) > 2e8
    B = Batch(mats)
    ys = [torch.empty(A.n_rows, dtype=tdt, device="cuda") for A in As]
    xd = [torch.empty(A.n_cols, dtype=tdt, device="cuda") for A in As]
    for rep in range(2):  # same buffers: the second apply replays the captured graph
        xs = [W.uniform(A.n_cols, 1000 * rep + m).astype(npdt) for m, A in enumerate(As)]
        for m in range(len(As)):
            xd[m].copy_(torch.as_tensor(xs[m]))
        B.apply(xd, ys)
        torch.cuda.synchronize()
        for m, A in enumerate(As):
            ref, bound = oracle.spmv(A.row_ptr, A.col_idx, A.val.astype(npdt).astype(np.float64),
                                     xs[m].astype(np.float64), with_bound=True)
            assert_within(host(ys[m]), ref, bound, rel, f"batch {dtype} m={m} rep={rep}")


@pytest.mark.parametrize("dtype", ["f64", "f32"])
def test_batched_follows_member_values(dtype):
    """New values set on one member handle after the batch was built reach the
    next batched launch (the batch lays that member's values out again)."""
    from paper_1106_5908_gb300 import Batch, Matrix
    As = [W.batch_matrix(m, n, seed=9) for m, n in enumerate((3000, 5000, 800, 12000))]
    npdt = np.float32 if dtype == "f32" else np.float64
    mats = [Matrix.from_csr(A.row_ptr, A.col_idx, A.val.astype(npdt), A.n_cols) for A in As]
    B = Batch(mats)
    xs = [W.uniform(A.n_cols, 60 + m).astype(npdt) for m, A in enumerate(As)]
    xd = [dev(x) for x in xs]
    ys = [torch.zeros(A.n_rows, dtype=xd[0].dtype, device="cuda") for A in As]
    B.apply(xd, ys)
    v2 = W.uniform(As[2].nnz, 61).astype(npdt)
    mats[2].set_values(dev(v2))
    B.apply(xd, ys)
    torch.cuda.synchronize()
    rel = 1e-6 if dtype == "f32" else 1e-13
    for m, A in enumerate(As):
        val = v2 if m == 2 else A.val.astype(npdt)
        ref, bound = oracle.spmv(A.row_ptr, A.col_idx, val.astype(np.float64), xs[m].astype(np.float64),
                                 with_bound=True)
        assert_within(host(ys[m]), ref, bound, rel, f"member {m}")


def test_batched_integer_bitexact():
    from paper_1106_5908_gb300 import Batch, Matrix
    As = [W.random_csr(n, n, seed=n, integer=True, max_len=20, long_rows=1, long_len=min(n, 4000))
          for n in (100, 3000, 5000, 17)]
    B = Batch([Matrix.from_csr(A.row_ptr, A.col_idx, A.val, A.n_cols) for A in As])
    xs = [W.integers(A.n_cols, A.n_rows) for A in As]
    ys = [torch.zeros(A.n_rows, dtype=torch.float64, device="cuda") for A in As]
    B.apply([dev(x) for x in xs], ys)
    for A, x, y in zip(As, xs, ys):
        assert_bitexact(host(y), oracle.spmv(*A.astuple(), x))
