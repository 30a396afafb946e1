"""The pins catch plausible mistakes: each case copies the oracle's C source,
plants one mistake (a dropped term, a wrong sign or index, a transposed operand,
an off-by-one), compiles the copy on the CPU, swaps it in, and checks that at
least one pin of tests/test_oracle_pins.py fails."""
import contextlib
import ctypes
import os
import subprocess
import tempfile

import pytest

import oracle
import test_oracle_node_pins as npins
import test_oracle_pins as pins

FUNCS = ("oracle_spmv", "oracle_spmv_omp", "oracle_num_threads", "oracle_spmm", "oracle_transpose",
         "oracle_backward", "oracle_split_blocks", "oracle_split_halo", "oracle_cg",
         "oracle_row_histogram", "oracle_thread_rows", "oracle_spmv_f32", "oracle_spmv_split",
         "oracle_node_create", "oracle_node_destroy", "oracle_node_spmv", "oracle_node_spmv_f32",
         "oracle_node_spmv_split", "oracle_node_set_y", "oracle_node_get_y", "oracle_node_threads",
         "oracle_spmv_sym")


@contextlib.contextmanager
def planted(old: str, new: str):
    real = oracle._load()
    src = open(oracle._SRC).read()
    assert src.count(old) >= 1, f"mutation site not found: {old!r}"
    src = src.replace(old, new, 1)
    with tempfile.TemporaryDirectory() as d:
        c = os.path.join(d, "mutant.c")
        so = os.path.join(d, "libmutant.so")
        open(c, "w").write(src)
        subprocess.run(["gcc", "-O1", "-ffp-contract=off", "-fopenmp", "-fPIC", "-shared", "-o", so, c, "-lm"],
                       check=True)
        lib = ctypes.CDLL(so)
        for f in FUNCS:
            getattr(lib, f).argtypes = getattr(real, f).argtypes
            getattr(lib, f).restype = getattr(real, f).restype
        oracle._lib = lib
        try:
            yield
        finally:
            oracle._lib = real


SPMV_PINS = [
    lambda: pins.test_spmv_vs_dense_and_scipy((17, 33), 1),
    lambda: pins.test_laplace2d_closed_forms(5, 5),
    lambda: pins.test_laplace3d_closed_forms(6),
    lambda: pins.test_dirichlet_eigenpairs(2, 12, (3, 7)),
    lambda: pins.test_integer_exact(1),
    lambda: pins.test_empty_rows_give_beta_y(),
    lambda: pins.test_one_based_listing_reading(),
]

OMP_PINS = [
    lambda: npins.test_spmv_omp_equals_plain_bit_for_bit((17, 33), 3),
    lambda: npins.test_spmv_omp_equals_plain_bit_for_bit((301, 301), 0),
    lambda: npins.test_spmv_omp_hamiltonian_like(3),
    lambda: npins.test_thread_rows_is_the_nonzero_balanced_rule(4, 1),
]
NODE_PINS = [
    lambda: npins.test_first_touch_node_equals_the_plain_forms((301, 301), 3, 8),
    lambda: npins.test_first_touch_node_hamiltonian_like(),
]
SPLIT_PINS = [
    lambda: npins.test_spmv_split_literal_and_plain((64, 64), 3),
    lambda: npins.test_spmv_split_integer_exact(),
]

SYM_PINS = [
    lambda: pins.test_spmv_sym_vs_dense_and_full(64, 1),
    lambda: pins.test_spmv_sym_integer_exact_and_laplacians(),
]

MUTANTS = {
    # Listing 1 kernel
    "drop the last entry of each row": (
        "for (int32_t k = row_ptr[i]; k < row_ptr[i + 1]; ++k) {\n            double p = val[k] * x[col_idx[k]];",
        "for (int32_t k = row_ptr[i]; k < row_ptr[i + 1] - 1; ++k) {\n            double p = val[k] * x[col_idx[k]];",
        SPMV_PINS),
    "skip the first entry of each row": (
        "for (int32_t k = row_ptr[i]; k < row_ptr[i + 1]; ++k) {\n            double p = val[k] * x[col_idx[k]];",
        "for (int32_t k = row_ptr[i] + 1; k < row_ptr[i + 1]; ++k) {\n            double p = val[k] * x[col_idx[k]];",
        SPMV_PINS),
    "wrong sign in the row sum": ("acc = acc + p;\n            mag", "acc = acc - p;\n            mag", SPMV_PINS),
    "row index instead of column": ("double p = val[k] * x[col_idx[k]];\n            acc = acc + p;\n            mag",
                                    "double p = val[k] * x[i < 0 ? 0 : i];\n            acc = acc + p;\n            mag",
                                    SPMV_PINS),
    "beta dropped": ("y[i] = alpha * acc + beta * yin;", "y[i] = alpha * acc + yin;", SPMV_PINS),
    "alpha dropped": ("y[i] = alpha * acc + beta * yin;", "y[i] = acc + beta * yin;", SPMV_PINS),
    # block vectors
    "block vectors read the wrong column": ("X[(int64_t)col_idx[k] * nrhs + r]", "X[(int64_t)col_idx[k] * nrhs]",
                                            [lambda: pins.test_spmm_vs_dense(4), lambda: pins.test_spmm_vs_dense(8)]),
    # transpose
    "transpose counts one column off": ("rowT_ptr[col_idx[k] + 1] += 1;", "rowT_ptr[col_idx[k]] += 1;",
                                        [lambda: pins.test_transpose_vs_scipy((40, 30), False),
                                         lambda: pins.test_transpose_twice_is_identity()]),
    "transpose records the column, not the row": ("colT_idx[p] = i;", "colT_idx[p] = col_idx[k];",
                                                  [lambda: pins.test_transpose_vs_scipy((40, 30), False),
                                                   lambda: pins.test_transpose_twice_is_identity()]),
    # reverse pass
    "grad_val with g and x swapped": ("grad_val[k] = alpha * (g[i] * x[col_idx[k]]);",
                                      "grad_val[k] = alpha * (g[col_idx[k] % n_rows] * x[i % n_cols]);",
                                      [lambda: pins.test_backward_vs_dense_and_fd(1)]),
    "grad_x scattered to the row": ("acc[col_idx[k]] = acc[col_idx[k]] + p;",
                                    "acc[i % n_cols] = acc[i % n_cols] + p;",
                                    [lambda: pins.test_backward_vs_dense_and_fd(1)]),
    # split bookkeeping (Sect. 3.2)
    "block start uses <= instead of <": ("while (r < n_rows && row_ptr[r] < target)",
                                         "while (r < n_rows && row_ptr[r] <= target)",
                                         [lambda: pins.test_split_blocks_definition(3, 1),
                                          lambda: pins.test_split_blocks_definition(8, 5)]),
    "halo keeps local columns": ("if (j >= lo && j < hi) {\n                    ++nl;",
                                 "if (j >= lo && j < hi) {\n                    used[j] = 1;\n                    ++nl;",
                                 [lambda: pins.test_split_halo_brute_force(4)]),
    # node-level loop (Sect. 2 / 3.5 explicit distribution)
    "node-level loop drops the last entry of each row": (
        "for (int32_t k = row_ptr[i]; k < row_ptr[i + 1]; ++k)\n            acc = acc + val[k] * x[col_idx[k]];",
        "for (int32_t k = row_ptr[i]; k < row_ptr[i + 1] - 1; ++k)\n            acc = acc + val[k] * x[col_idx[k]];",
        OMP_PINS),
    "node-level loop drops beta": ("y[i] = alpha * acc + beta * y[i];", "y[i] = alpha * acc + y[i];", OMP_PINS),
    "thread chunk skips its first row": ("spmv_rows(bounds[t], bounds[t + 1], row_ptr",
                                         "spmv_rows(bounds[t] + (t > 0), bounds[t + 1], row_ptr", OMP_PINS),
    "thread chunks round the nonzero target down": ("((int64_t)t * nnz + nthreads - 1) / nthreads",
                                                    "((int64_t)t * nnz) / nthreads", OMP_PINS),
    "FP32 form sums in float": ("acc = acc + (double)val[k] * (double)x[col_idx[k]];",
                                "acc = (float)(acc + (float)((float)val[k] * (float)x[col_idx[k]]));",
                                [lambda: npins.test_spmv_f32_is_the_upcast_product_rounded_once((200, 150), 1)]),
    "first-touch copy forgets the last row offset": ("nd->rp[n_rows] = row_ptr[n_rows];", "(void)0;", NODE_PINS),
    "node FP32 form reads the FP64 values": ("acc = acc + (double)nd->val32[k] * (double)nd->x32[nd->ci[k]];",
                                             "acc = acc + nd->val[k] * nd->x[nd->ci[k]];", NODE_PINS),
    # split form (Sect. 3.4)
    "split nonlocal part applies beta again": ("y[i] = y[i] + alpha * acc;", "y[i] = beta * y[i] + alpha * acc;",
                                               SPLIT_PINS),
    "split local test includes the block end": ("if (j >= lo && j < hi)\n                    acc = acc + val[k] * x[j];",
                                                "if (j >= lo && j <= hi)\n                    acc = acc + val[k] * x[j];",
                                                SPLIT_PINS),
    "node split reads the halo one position off": ("acc = acc + nd->valn[k] * nd->halo[nd->cin[k]];",
                                                   "acc = acc + nd->valn[k] * nd->halo[nd->cin[k] > 0 ? nd->cin[k] - 1 : 0];",
                                                   NODE_PINS),
    # symmetric CRS (Sect. 1.3.1)
    "symmetric form counts the diagonal twice": ("            if (j != i) {\n                double q = val[k] * x[i];",
                                                 "            if (1) {\n                double q = val[k] * x[i];",
                                                 SYM_PINS),
    "symmetric form mirrors with x[j]": ("double q = val[k] * x[i];", "double q = val[k] * x[j];", SYM_PINS),
    "symmetric form drops the mirrored entry": ("                t[j] = t[j] + q;", "                t[j] = t[j] + 0.0 * q;",
                                                SYM_PINS),
    # CG
    "CG update with the wrong sign": ("r[i] = r[i] - a * q[i];", "r[i] = r[i] + a * q[i];",
                                      [lambda: pins.test_cg_solves_spd()]),
}


def _run_mutant(name, q):
    old, new, checks = MUTANTS[name]
    caught = 0
    with planted(old, new):
        for chk in checks:
            try:
                chk()
            except Exception:  # an assertion (or any error) of a pin catches the mistake
                caught += 1
    q.put(caught)


@pytest.mark.parametrize("name", list(MUTANTS))
def test_planted_mistake_is_caught(name):
    """Each planted copy runs in a child process: a mistake that makes the copy
    write out of bounds kills only the child, which also counts as caught."""
    import multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    p = ctx.Process(target=_run_mutant, args=(name, q))
    p.start()
    p.join(timeout=300)
    if p.exitcode == 0:
        caught = q.get(timeout=10)
        assert caught > 0, f"no pin failed for planted mistake: {name}"
    else:
        assert p.exitcode is not None, "planted copy did not finish"


def test_unplanted_oracle_passes_the_same_checks():
    for _, _, checks in MUTANTS.values():
        for chk in checks:
            chk()
