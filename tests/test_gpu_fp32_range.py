"""FP32-stored operands whose products leave FP32's range, against the oracle
(exact products of the floats summed in FP64: FP32 storage with FP64
accumulation).  Every FP32 plan with both accumulators, FP32 and FP64 results
and every alpha/beta form; the reverse pass (first pass through the
permutation, second on the laid-out copy of A^T), the batched launch and the
IR-CG inner solve on such data.

The float-float accumulator marks a row whose products it cannot split exactly
(a nonzero product below 2^-100, an overflow, an inf or NaN operand) and that
row is summed again with FP64 products, so each result must meet the
FP32-storage bound 1e-6 * sum_j |a_ij x_j|; an FP32 result may in addition
differ from the exact value by the rounding to float itself (which alone
exceeds the bound for results in FP32's subnormal range); infinities and NaN
must match the oracle's."""
import numpy as np
import pytest

import oracle
from paper_1106_5908_gb300 import workloads as W
from gpu_util import dev, host, need_gpu

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

PLANS = [(6, 9), (6, 15), (0, 15), (0, 7), (3, 15), (4, 7), (4, 9), (4, 15), (5, 32), (5, 256), (5, 4096), (0, 16),
         (2, 15), (2, 31), (1, 1), (1, 4), (1, 32)]
FORMS = [(1.0, 0.0), (-0.75, 1.0), (2.0, -0.5), (1.0, 1.0)]


@pytest.fixture(autouse=True)
def _gpu():
    need_gpu()


def check(y, ref, bound, out32, what):
    y = np.asarray(y, dtype=np.float64)
    ref = np.asarray(ref, dtype=np.float64)
    nan = np.isnan(ref)
    bad = np.flatnonzero(np.isnan(y) != nan)
    assert bad.size == 0, f"{what}: NaN differs at {bad[:5]}: got {y[bad[:5]]}, want {ref[bad[:5]]}"
    want = ref.astype(np.float32).astype(np.float64) if out32 else ref
    inf = np.isinf(want) & ~nan
    bad = np.flatnonzero(inf & (y != want))
    assert bad.size == 0, f"{what}: infinity differs at {bad[:5]}: got {y[bad[:5]]}, want {want[bad[:5]]}"
    ok = ~nan & ~inf
    lim = 1e-6 * bound[ok] + (np.abs(want[ok] - ref[ok]) if out32 else 0.0)
    err = np.abs(y[ok] - ref[ok])
    bad = np.flatnonzero(~(err <= lim))
    assert bad.size == 0, (f"{what}: {bad.size} rows outside the bound; first: got {y[ok][bad[:5]]}, "
                           f"want {ref[ok][bad[:5]]}, bound {lim[bad[:5]]}")


def make32(A):
    from paper_1106_5908_gb300 import Matrix
    return Matrix.from_csr(A.row_ptr, A.col_idx, A.val.astype(np.float32), A.n_cols)


def logu(rng, n, lo=-149.0, hi=127.0):
    mag = np.exp2(rng.uniform(lo, hi, n))
    return (mag * np.where(rng.random(n) < 0.5, -1.0, 1.0)).astype(np.float32)


@pytest.mark.parametrize("acc", ["ff", "f64"])
@pytest.mark.parametrize("plan", PLANS)
def test_fp32_range_every_plan(plan, acc):
    A, x = W.fp32_range_case()
    M = make32(A)
    M.set_accumulator(acc)
    M.set_plan(*plan)
    v64 = A.val.astype(np.float64)
    y0 = W.uniform(A.n_rows, 17).astype(np.float32)
    for out in (torch.float32, torch.float64):
        out32 = out == torch.float32
        for alpha, beta in FORMS:
            yin = y0 if out32 else y0.astype(np.float64)
            ref, bound = oracle.spmv(A.row_ptr, A.col_idx, v64, x.astype(np.float64), alpha, beta,
                                     yin.astype(np.float64), with_bound=True)
            y = dev(yin)
            M.apply(dev(x), y, alpha, beta)
            check(host(y), ref, bound, out32, f"plan {plan} acc {acc} out {out} a={alpha} b={beta}")


@pytest.mark.parametrize("acc", ["ff", "f64"])
def test_fp32_widening_of_every_class(acc):
    """With a unit diagonal y_i = x_i exactly, for zeros, subnormals, the ends of
    the normal range, infinities and NaN (both accumulators)."""
    rng = np.random.default_rng(5)
    bits = np.concatenate([
        np.array([0x00000000, 0x80000000, 0x00000001, 0x80000001, 0x007fffff, 0x807fffff, 0x00400000,
                  0x00800000, 0x80800000, 0x7f7fffff, 0xff7fffff, 0x3f800000, 0x33800000,
                  0x7f800000, 0xff800000, 0x7fc00000, 0x7fa00001], np.uint32),
        rng.integers(1, 0x00800000, 64, dtype=np.uint32),
        rng.integers(0x00800000, 0x7f800000, 256, dtype=np.uint32) | (rng.integers(0, 2, 256, dtype=np.uint32) << 31)])
    x32 = bits.view(np.float32)
    n = x32.size
    A = W.CRS(np.arange(n + 1, dtype=np.int32), np.arange(n, dtype=np.int32), np.ones(n, np.float32), n)
    for plan in PLANS:
        M = make32(A)
        M.set_accumulator(acc)
        M.set_plan(*plan)
        y = host(M.apply(dev(x32), out_dtype=torch.float64))
        want = x32.astype(np.float64)
        nan = np.isnan(want)
        assert np.array_equal(np.isnan(y), nan), plan
        assert np.array_equal(y[~nan], want[~nan]), (plan, np.flatnonzero(y[~nan] != want[~nan])[:8])


def test_fp32_range_full_size_slot_kernel():
    """The Hamiltonian-like matrix at full size in FP32 storage, one value in
    every 4096 entries scaled to 1e-30 and one x entry in every 4096 scaled to
    1e25 (products below 2^-100 and above 2^64 spread over every chunk), against
    the oracle on every row."""
    A = W.hamiltonian_like(W.HAMILTONIAN_N, seed=W.SEED_HAMILTONIAN)
    v32 = A.val.astype(np.float32)
    v32[::4096] *= np.float32(1e-30)
    x32 = W.uniform(A.n_cols, W.SEED_HAMILTONIAN_X).astype(np.float32)
    x32[7::4096] *= np.float32(1e25)
    from paper_1106_5908_gb300 import Matrix
    M = Matrix.from_csr(A.row_ptr, A.col_idx, v32, A.n_cols)
    assert M.info()["family"] == 4
    ref, bound = oracle.spmv(A.row_ptr, A.col_idx, v32.astype(np.float64), x32.astype(np.float64), with_bound=True)
    check(host(M.apply(dev(x32))), ref, bound, True, "Hamiltonian-like FP32, FP32 y")
    check(host(M.apply(dev(x32), out_dtype=torch.float64)), ref, bound, False, "Hamiltonian-like FP32, FP64 y")


def _stencil_wild(seed):
    A = W.stencil27(12, seed=seed)
    rng = np.random.default_rng(seed)
    v = logu(rng, A.nnz, -80.0, 60.0)
    return W.CRS(A.row_ptr, A.col_idx, v, A.n_cols), rng


@pytest.mark.parametrize("kind", ["scattered", "stencil"])
def test_fp32_range_reverse_pass(kind):
    """grad_x = alpha*A^T g and grad_val on FP32 storage with products out of
    FP32's range: the first reverse pass (values through the permutation) and
    the second (values laid out in A^T order: the slot-major copy of A^T for
    scattered columns, the row-slice copy for the 27-point pattern)."""
    if kind == "scattered":
        A, x = W.fp32_range_case(special=False)
        rng = np.random.default_rng(3)
    else:
        A, rng = _stencil_wild(4)
        x = logu(rng, A.n_cols, -80.0, 60.0)
    g = logu(rng, A.n_rows, -80.0, 60.0)
    M = make32(A)
    v64 = A.val.astype(np.float64)
    for alpha in (1.0, -0.5):
        gx_ref, gv_ref, bgx = oracle.backward(A.row_ptr, A.col_idx, v64, A.n_cols, g.astype(np.float64),
                                              x.astype(np.float64), alpha, with_bound=True)
        for rep in range(2):
            gx, gv = M.backward(dev(g), dev(x), alpha)
            check(host(gx), gx_ref, bgx, True, f"{kind} grad_x pass {rep} alpha {alpha}")
            check(host(gv), gv_ref, np.abs(gv_ref), True, f"{kind} grad_val pass {rep} alpha {alpha}")


def test_fp32_range_batched():
    from paper_1106_5908_gb300 import Batch
    cases = [W.fp32_range_case(seed=s, n_normal=n) for s, n in ((1, 500), (2, 3000), (3, 50))]
    A4, rng = _stencil_wild(5)
    cases.append((A4, logu(rng, A4.n_cols, -80.0, 60.0)))
    mats = [make32(A) for A, _ in cases]
    B = Batch(mats)
    for rep in range(2):
        ys = [torch.zeros(A.n_rows, dtype=torch.float32, device="cuda") for A, _ in cases]
        B.apply([dev(x) for _, x in cases], ys)
        torch.cuda.synchronize()
        for m, (A, x) in enumerate(cases):
            ref, bound = oracle.spmv(A.row_ptr, A.col_idx, A.val.astype(np.float64), x.astype(np.float64),
                                     with_bound=True)
            check(host(ys[m]), ref, bound, True, f"batch member {m} rep {rep}")


@pytest.mark.parametrize("scale", [1.0, 1e-35])
def test_ir_cg_inner_solve_out_of_range(scale):
    """IR-CG on a 7-point Poisson matrix scaled by 1e-35: the FP32 inner solve's
    products (matrix values ~6e-35 times unit-norm vectors) and dot products fall
    below 2^-100, so they take the FP64 path; the solve must converge as the
    unscaled one does, with the residual rechecked by the oracle."""
    from paper_1106_5908_gb300 import Matrix, ir_cg
    A = W.laplace3d(16)
    As = W.CRS(A.row_ptr, A.col_idx, A.val * scale, A.n_cols)
    M = Matrix.from_csr(As.row_ptr, As.col_idx, As.val, As.n_cols)
    b = W.uniform(A.n_rows, 77) * scale
    x, st = ir_cg(M, dev(b), outer_tol=1e-12, max_outer=50)
    assert st["converged"], st
    r = oracle.residual(*As.astuple(), b, host(x))
    assert np.linalg.norm(r) / np.linalg.norm(b) <= 1.5e-12, st
    assert st["outer"] <= 8, st
