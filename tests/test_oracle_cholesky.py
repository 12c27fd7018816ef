"""Pins for the oracle's Cholesky factor (the map R = mu + C z of the normal
law in Sec. 3.1 needs C with C C' = Sigma).

Checked against a hand-computed integer example, LAPACK's factor through
numpy, the reconstruction C C' = Sigma, the diagonal special case, that only
the lower triangle of Sigma is read, and the rejection of an indefinite
matrix."""
import numpy as np
import pytest

import oracle
from paper_2404_11631_gb300 import inputs


def test_hand_computed_example_is_exact():
    # C00 = 2, C10 = 2/2, C11 = sqrt(10 - 1), C20 = -2/2,
    # C21 = (2 - (-1)(1)) / 3, C22 = sqrt(6 - 1 - 1)
    S = np.array([[4.0, 2.0, -2.0], [2.0, 10.0, 2.0], [-2.0, 2.0, 6.0]])
    C = oracle.cholesky(S)
    assert np.array_equal(C, np.array([[2.0, 0.0, 0.0], [1.0, 3.0, 0.0], [-1.0, 1.0, 2.0]]))


@pytest.mark.parametrize("d", [1, 2, 7, 64, 200])
def test_matches_lapack_and_reconstructs(d):
    S = inputs.instance(d, seed=d).sigma
    C = oracle.cholesky(S)
    ref = np.linalg.cholesky(S)
    assert np.max(np.abs(C - ref)) <= 1e-12 * np.max(np.abs(ref))
    assert np.array_equal(np.triu(C, 1), np.zeros((d, d)))
    assert np.max(np.abs(C @ C.T - S)) <= 1e-13 * np.max(np.abs(S))
    assert np.all(np.diag(C) > 0)


def test_diagonal_sigma_gives_square_roots():
    v = np.array([0.25, 2.0, 1e-6, 9.0, 3.0])
    C = oracle.cholesky(np.diag(v))
    assert np.array_equal(C, np.diag(np.sqrt(v)))


def test_upper_triangle_is_not_read():
    S = inputs.instance(16, seed=3).sigma
    T = np.tril(S) + np.triu(np.full((16, 16), 1e300), 1)
    assert np.array_equal(oracle.cholesky(T), oracle.cholesky(S))


def test_indefinite_matrix_is_rejected():
    with pytest.raises(ValueError):
        oracle.cholesky(np.array([[1.0, 2.0], [2.0, 1.0]]))
    with pytest.raises(ValueError):
        oracle.cholesky(np.zeros((3, 3)))
