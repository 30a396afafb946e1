"""The input generators' structural helpers: the orderings of the ordering study
(P A P^T against a dense permutation, RCM on a scrambled stencil) and the Hamiltonian-like
recipe's shape."""
import numpy as np
import pytest

from paper_1106_5908_gb300 import workloads as W


def dense(A):
    D = np.zeros((A.n_rows, A.n_cols))
    rows = np.repeat(np.arange(A.n_rows), np.diff(A.row_ptr))
    np.add.at(D, (rows, A.col_idx), A.val)
    return D


@pytest.mark.parametrize("seed", [0, 1])
def test_permute_symmetric_is_pap(seed):
    A = W.hamiltonian_like(300, seed=seed + 10)
    order = W.random_order(A.n_rows, seed)
    B = W.permute_symmetric(A, order)
    D = dense(A)
    np.testing.assert_array_equal(dense(B), D[np.ix_(order, order)])
    assert B.nnz == A.nnz
    for i in range(B.n_rows):  # columns sorted within rows
        c = B.col_idx[B.row_ptr[i]:B.row_ptr[i + 1]]
        assert np.all(np.diff(c) > 0)


def test_rcm_recovers_a_band():
    """A 2D 5-point Laplacian (bandwidth nx) scrambled by a random ordering has a
    bandwidth near n; RCM brings it back to the order of nx."""
    A = W.laplace2d(40, 40)
    assert W.bandwidth(A) == 40
    S = W.permute_symmetric(A, W.random_order(A.n_rows, 3))
    assert W.bandwidth(S) > 1000
    order = W.rcm_order(S)
    assert np.array_equal(np.sort(order), np.arange(S.n_rows))
    assert W.bandwidth(W.permute_symmetric(S, order)) <= 2 * 40


def test_hamiltonian_like_recipe_small():
    """Upper rows: ceil(l/2) columns within (i, i+64], floor(l/2) beyond; mirrored
    with a diagonal, so the pattern is symmetric."""
    A = W.hamiltonian_like(5000, seed=1)
    D = dense(A)
    assert np.array_equal(D != 0, (D != 0).T)
    assert np.all(np.diag(D) != 0) or np.count_nonzero(np.diag(D) == 0) < 5
    near = far = 0
    rows = np.repeat(np.arange(A.n_rows), np.diff(A.row_ptr))
    up = A.col_idx > rows
    d = A.col_idx[up] - rows[up]
    near, far = int(np.sum(d <= 64)), int(np.sum(d > 64))
    assert 0.9 < near / far < 1.6
