"""GPU parity on the Hamiltonian-like matrix at full size (N = 4,194,304): plain
FP64, the local/nonlocal split over 8 nonzero-balanced or equal-rows blocks (plan
and halo bit-exact, result within tolerance, in task mode on two streams, naive
overlap on one stream, and vector mode), FP32 storage, and block vectors."""
import numpy as np
import pytest

import oracle
from paper_1106_5908_gb300 import workloads as W
from gpu_util import assert_bitexact, assert_within, dev, host, need_gpu

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def ham():
    need_gpu()
    A = W.hamiltonian_like(W.HAMILTONIAN_N, seed=W.SEED_HAMILTONIAN)
    x = W.uniform(A.n_rows, W.SEED_HAMILTONIAN_X)
    ref, bound = oracle.spmv(*A.astuple(), x, with_bound=True)
    return A, x, ref, bound


@pytest.fixture(scope="module")
def m_ham(ham):
    from paper_1106_5908_gb300 import Matrix
    A = ham[0]
    return Matrix.from_csr(A.row_ptr, A.col_idx, A.val, A.n_cols)


def test_hamiltonian_shape(ham):
    A = ham[0]
    assert A.n_rows == 4194304
    assert 12.5 < A.nnz / A.n_rows < 13.5


def test_hamiltonian_plain_f64(ham, m_ham):
    A, x, ref, bound = ham
    y = m_ham.apply(dev(x))
    assert_within(host(y), ref, bound, 1e-13, "Hamiltonian plain")
    # alpha/beta update on the same launch shape
    y0 = W.uniform(A.n_rows, 77)
    ref2, bound2 = oracle.spmv(*A.astuple(), x, -2.0, 0.5, y0, with_bound=True)
    y = dev(y0)
    m_ham.apply(dev(x), y, -2.0, 0.5)
    assert_within(host(y), ref2, bound2, 1e-13, "Hamiltonian alpha/beta")


@pytest.mark.parametrize("plan", [(6, 7), (6, 9), (0, 15), (0, 7), (3, 7), (3, 15), (4, 7), (4, 9), (4, 11), (4, 15),
                                  (5, 256), (5, 4096), (0, 16), (0, 8), (2, 7), (2, 15), (2, 31), (1, 2)])
def test_hamiltonian_plans(ham, m_ham, plan):
    A, x, ref, bound = ham
    m_ham.set_plan(*plan)
    try:
        assert_within(host(m_ham.apply(dev(x))), ref, bound, 1e-13, f"Hamiltonian plan={plan}")
    finally:
        m_ham.set_plan(0, 16)


def test_hamiltonian_split(ham, m_ham):
    A, x, ref, bound = ham
    sp = m_ham.split(8)
    plan = sp.plan()
    bs = oracle.split_blocks(A.row_ptr, 8)
    assert_bitexact(plan["block_start"], bs, "block starts")
    cnt, hmap, nl, nn = oracle.split_halo(A.row_ptr, A.col_idx, A.n_cols, bs)
    assert_bitexact(plan["halo_count"], cnt, "halo counts")
    assert_bitexact(plan["halo_map"], hmap, "halo map")
    assert_bitexact(plan["nnz_local"], nl, "local entries")
    assert_bitexact(plan["nnz_nonlocal"], nn, "nonlocal entries")
    xd = dev(x)
    s1 = torch.cuda.Stream()
    s2 = torch.cuda.Stream()
    for s_comm in (None, s2):  # one stream (naive overlap) and two streams
        y = sp.apply(xd, s_compute=s1, s_comm=s_comm)
        s1.synchronize()
        assert_within(host(y), ref, bound, 1e-13, f"split comm={s_comm}")
        assert_bitexact(sp.halo(), x[hmap], "gathered halo")
    y0 = W.uniform(A.n_rows, 5)
    ref2, bound2 = oracle.spmv(*A.astuple(), x, 0.5, -1.0, y0, with_bound=True)
    y = dev(y0)
    sp.apply(xd, y, 0.5, -1.0, s_compute=s1, s_comm=s2)
    s1.synchronize()
    assert_within(host(y), ref2, bound2, 1e-13, "split alpha/beta")


@pytest.mark.parametrize("equal_rows", [False, True])
def test_hamiltonian_split_vector_mode(ham, m_ham, equal_rows):
    """Vector mode (Fig. kernel_schemes (a)) gives the plain product; equal-rows
    blocks start at floor(b*n/8)."""
    A, x, ref, bound = ham
    sp = m_ham.split(8, equal_rows=equal_rows)
    plan = sp.plan()
    if equal_rows:
        assert_bitexact(plan["block_start"], np.array([b * A.n_rows // 8 for b in range(9)]), "equal rows")
    cnt, hmap, _, _ = oracle.split_halo(A.row_ptr, A.col_idx, A.n_cols, plan["block_start"])
    assert_bitexact(plan["halo_map"], hmap, "halo map")
    xd = dev(x)
    assert_within(host(sp.apply_vector(xd)), ref, bound, 1e-13, "vector mode")
    assert_within(host(sp.apply(xd, s_comm=torch.cuda.Stream())), ref, bound, 1e-13, "task mode")
    torch.cuda.synchronize()
    y0 = W.uniform(A.n_rows, 6)
    ref2, bound2 = oracle.spmv(*A.astuple(), x, -1.5, 0.25, y0, with_bound=True)
    y = dev(y0)
    sp.apply_vector(xd, y, -1.5, 0.25)
    assert_within(host(y), ref2, bound2, 1e-13, "vector mode alpha/beta")


def test_split_vector_mode_small_and_integer():
    """Vector mode on explicit blocks (one empty), one block (no halo) and
    integer data (bit-exact)."""
    from paper_1106_5908_gb300 import Matrix
    A = W.hamiltonian_like(5000, seed=4)
    M = Matrix.from_csr(A.row_ptr, A.col_idx, A.val, A.n_cols)
    x = W.uniform(5000, 1)
    ref, bound = oracle.spmv(*A.astuple(), x, with_bound=True)
    for starts in ([0, 100, 100, 2500, 4999, 5000], [0, 5000]):
        sp = M.split(len(starts) - 1, starts)
        assert_within(host(sp.apply_vector(dev(x))), ref, bound, 1e-13, f"vector mode {starts}")
    assert M.split(1).plan()["total_halo"] == 0
    Ai = W.random_csr(3000, 3000, seed=8, integer=True, max_len=30)
    Mi = Matrix.from_csr(Ai.row_ptr, Ai.col_idx, Ai.val, Ai.n_cols)
    xi = W.integers(3000, 9).astype(np.float64)
    refi = oracle.spmv(*Ai.astuple(), xi)
    for eq in (False, True):
        spi = Mi.split(8, equal_rows=eq)
        assert_bitexact(host(spi.apply_vector(dev(xi))), refi, f"vector mode integer eq={eq}")
        y = spi.apply(dev(xi), s_comm=torch.cuda.Stream())
        torch.cuda.synchronize()
        assert_bitexact(host(y), refi, f"task mode integer eq={eq}")


def test_split_explicit_blocks_small():
    from paper_1106_5908_gb300 import Matrix
    A = W.hamiltonian_like(5000, seed=4)
    M = Matrix.from_csr(A.row_ptr, A.col_idx, A.val, A.n_cols)
    starts = [0, 100, 100, 2500, 4999, 5000]  # includes an empty block
    sp = M.split(5, starts)
    plan = sp.plan()
    cnt, hmap, nl, nn = oracle.split_halo(A.row_ptr, A.col_idx, A.n_cols, np.array(starts, np.int32))
    assert_bitexact(plan["halo_map"], hmap)
    assert_bitexact(plan["halo_count"], cnt)
    x = W.uniform(5000, 1)
    ref, bound = oracle.spmv(*A.astuple(), x, with_bound=True)
    y = sp.apply(dev(x), s_comm=torch.cuda.Stream())
    torch.cuda.synchronize()
    assert_within(host(y), ref, bound, 1e-13)


@pytest.mark.parametrize("plan", [None, (6, 9), (6, 15)])
@pytest.mark.parametrize("acc", ["ff", "f64"])
def test_hamiltonian_fp32_storage(ham, acc, plan):
    from paper_1106_5908_gb300 import Matrix
    A, x, _, _ = ham
    v32 = A.val.astype(np.float32)
    x32 = x.astype(np.float32)
    M = Matrix.from_csr(A.row_ptr, A.col_idx, v32, A.n_cols)
    M.set_accumulator(acc)
    if plan is not None:
        M.set_plan(*plan)
    ref, bound = oracle.spmv(A.row_ptr, A.col_idx, v32.astype(np.float64), x32.astype(np.float64),
                             with_bound=True)
    assert_within(host(M.apply(dev(x32))), ref, bound, 1e-6, f"Hamiltonian fp32 y32 {acc}")
    assert_within(host(M.apply(dev(x32), out_dtype=torch.float64)), ref, bound, 1e-6, f"Hamiltonian fp32 y64 {acc}")


@pytest.mark.parametrize("nrhs", [4, 8, 16, 32])
def test_hamiltonian_block_vectors(ham, m_ham, nrhs):
    """Block vectors on the full matrix, every row of Y against the oracle."""
    A, _, _, _ = ham
    X = W.uniform(0, W.SEED_BLOCK_X, shape=(A.n_rows, nrhs))
    Y = host(m_ham.spmm(dev(X)))
    ref, bound = oracle.spmm(*A.astuple(), X, with_bound=True)
    assert_within(Y.ravel(), ref.ravel(), bound.ravel(), 1e-13, f"Hamiltonian nrhs={nrhs}")
    # alpha/beta form on the same launch shape
    Y0 = W.uniform(0, 5, shape=(A.n_rows, nrhs))
    ref2, bound2 = oracle.spmm(*A.astuple(), X, -0.5, 2.0, Y0, with_bound=True)
    Yd = dev(Y0)
    m_ham.spmm(dev(X), Yd, -0.5, 2.0)
    assert_within(host(Yd).ravel(), ref2.ravel(), bound2.ravel(), 1e-13, f"Hamiltonian nrhs={nrhs} a/b")


@pytest.fixture(scope="module")
def reorderings(ham):
    A = ham[0]
    return {"rcm": W.rcm_order(A), "random": W.random_order(A.n_rows)}


@pytest.mark.parametrize("order", ["rcm", "random"])
def test_hamiltonian_reordered(ham, reorderings, order):
    """The ordering study's matrices (P A P^T in reverse Cuthill-McKee and in a
    random order, x permuted alike) through the autotuned plan, the row-slice
    plan, the split form and FP32 storage, against the oracle on the permuted
    matrix; the permuted product is the natural one permuted."""
    from paper_1106_5908_gb300 import Matrix
    A, x, ref_nat, _ = ham
    p = reorderings[order]
    B = W.permute_symmetric(A, p)
    xp = x[p]
    ref, bound = oracle.spmv(*B.astuple(), xp, with_bound=True)
    assert np.all(np.abs(ref - ref_nat[p]) <= 1e-13 * bound)
    M = Matrix.from_csr(B.row_ptr, B.col_idx, B.val, B.n_cols)
    info = M.info()
    assert_within(host(M.apply(dev(xp))), ref, bound, 1e-13, f"{order} auto {info['family']},{info['E']}")
    for plan in ((4, 7), (5, 4096)):
        M.set_plan(*plan)
        assert_within(host(M.apply(dev(xp))), ref, bound, 1e-13, f"{order} plan {plan}")
    sp = M.split(8)
    y = sp.apply(dev(xp), s_comm=torch.cuda.Stream())
    torch.cuda.synchronize()
    assert_within(host(y), ref, bound, 1e-13, f"{order} split")
    v32 = B.val.astype(np.float32)
    x32 = xp.astype(np.float32)
    M32 = Matrix.from_csr(B.row_ptr, B.col_idx, v32, B.n_cols)
    r32, b32 = oracle.spmv(B.row_ptr, B.col_idx, v32.astype(np.float64), x32.astype(np.float64), with_bound=True)
    assert_within(host(M32.apply(dev(x32))), r32, b32, 1e-6, f"{order} FP32")
