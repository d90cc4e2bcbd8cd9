"""Pins of the Hadamard transform and of the two embeddings."""
import numpy as np
import pytest
import scipy.linalg as sla

from oracle import hadamard, rng, sketch


@pytest.mark.parametrize("n", [1, 2, 8, 64, 512])
def test_hadamard_matches_sylvester_library(n):
    assert np.array_equal(hadamard.hadamard(n), sla.hadamard(n).astype(np.float64))


def test_hadamard_orthogonality():
    H = hadamard.hadamard(256)
    assert np.array_equal(H @ H.T, 256 * np.eye(256))


def test_fwht_equals_matrix_and_involution():
    x = np.random.default_rng(0).standard_normal((1024, 3))
    H = hadamard.hadamard(1024)
    y = hadamard.fwht(x)
    assert np.allclose(y, H @ x, rtol=0, atol=1e-10)
    assert np.allclose(hadamard.fwht(y), 1024 * x, rtol=0, atol=1e-9)
    with pytest.raises(ValueError):
        hadamard.fwht(np.ones(6))


def test_next_pow2():
    assert [hadamard.next_pow2(v) for v in (1, 2, 3, 4, 5, 4096, 4097)] == [1, 2, 4, 4, 8, 4096, 8192]


@pytest.mark.parametrize("n,m", [(100, 16), (128, 5), (257, 64)])
def test_srht_three_ways(n, m):
    """FWHT path, explicit-row sums and the dense S agree."""
    A = np.random.default_rng(n).standard_normal((n, 9))
    a = sketch.srht_sketch(A, m, seed=5, level=2)
    b = sketch.srht_rows_explicit(A, m, seed=5, level=2)
    c = sketch.srht_matrix(n, m, seed=5, level=2) @ A
    assert np.allclose(a, b, atol=1e-12) and np.allclose(a, c, atol=1e-12)


@pytest.mark.parametrize("n", [128, 100])
def test_srht_full_size_is_isometry(n):
    """m = n_pad keeps every row: S^T S = I_n exactly, so (SA)^T SA = A^T A."""
    n_pad = hadamard.next_pow2(n)
    S = sketch.srht_matrix(n, n_pad, seed=1, level=0)
    assert np.allclose(S.T @ S, np.eye(n), atol=1e-12)
    A = np.random.default_rng(1).standard_normal((n, 6))
    SA = sketch.srht_sketch(A, n_pad, seed=1, level=0)
    assert np.allclose(SA.T @ SA, A.T @ A, atol=1e-10)


def test_srht_unbiased():
    """E[S^T S] = I (Monte Carlo over seeds)."""
    n, m, trials = 32, 8, 1500
    acc = np.zeros((n, n))
    for s in range(trials):
        S = sketch.srht_matrix(n, m, seed=s, level=0)
        acc += S.T @ S
    acc /= trials
    # each column of S holds m entries of magnitude 1/sqrt(m): squared norm exactly 1
    assert np.abs(np.diag(acc) - 1).max() < 1e-12
    assert np.abs(acc - np.eye(n)).max() < 0.12


def test_gaussian_sketch_matches_dense():
    A = np.random.default_rng(2).standard_normal((300, 7))
    S = rng.gaussian_embedding(13, 300, seed=3, level=5)
    assert np.allclose(sketch.gaussian_sketch(A, 13, seed=3, level=5, block=64), S @ A, atol=1e-12)


def test_gaussian_unbiased():
    n, m, trials = 16, 4, 2000
    acc = np.zeros((n, n))
    for s in range(trials):
        S = rng.gaussian_embedding(m, n, seed=s, level=0)
        acc += S.T @ S
    acc /= trials
    assert np.abs(acc - np.eye(n)).max() < 0.12
