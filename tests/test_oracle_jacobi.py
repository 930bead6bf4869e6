"""Pins for the oracle's one-sided Jacobi SVD."""
import numpy as np
import pytest

from oracle.jacobi import jacobi_svd, svd_left


@pytest.mark.parametrize("m,k", [(1, 1), (5, 5), (9, 4), (33, 17), (64, 64)])
def test_matches_lapack_and_reconstructs(m, k):
    A = np.random.default_rng(m * 100 + k).standard_normal((m, k))
    U, s, V = jacobi_svd(A)
    ref = np.linalg.svd(A, compute_uv=False)
    assert np.abs(s - ref).max() <= 1e-13 * ref[0]
    assert np.abs((U * s) @ V.T - A).max() <= 1e-13 * ref[0]
    assert np.abs(V.T @ V - np.eye(k)).max() <= 1e-13
    assert np.abs(U.T @ U - np.eye(k)).max() <= 1e-12


def test_known_singular_values_graded():
    rng = np.random.default_rng(3)
    k = 12
    s_true = np.logspace(0, -11, k)
    Q1, _ = np.linalg.qr(rng.standard_normal((20, k)))
    Q2, _ = np.linalg.qr(rng.standard_normal((k, k)))
    A = (Q1 * s_true) @ Q2.T
    _, s, _ = jacobi_svd(A)
    assert np.abs(s - s_true).max() <= 1e-14


def test_rank_deficient_and_zero():
    A = np.zeros((6, 4))
    A[:, 0] = 1.0
    A[:, 2] = 2.0
    U, s, V = jacobi_svd(A)
    assert abs(s[0] - np.sqrt(6 * 5)) < 1e-13
    assert np.all(s[1:] < 1e-14)
    _, s0, _ = jacobi_svd(np.zeros((3, 3)))
    assert np.all(s0 == 0)


def test_svd_left_of_wide_matrix():
    F = np.random.default_rng(5).standard_normal((7, 40))
    W, s = svd_left(F)
    ref_u, ref_s, _ = np.linalg.svd(F)
    assert np.abs(s - ref_s).max() <= 1e-13 * ref_s[0]
    # same left subspaces (up to sign)
    assert np.abs(np.abs(np.sum(W * ref_u, axis=0)) - 1).max() <= 1e-10
