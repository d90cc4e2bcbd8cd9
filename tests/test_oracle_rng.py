"""Pins of the oracle's random draws: Philox known answers, distributions, and the
row-subset definition checked by brute force."""
import os

import numpy as np
import pytest
from scipy import stats

from oracle import philox, rng

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "philox4x32_10_kat.txt")


def _kat_rows():
    rows = []
    for line in open(GOLDEN):
        if line.startswith("#") or not line.strip():
            continue
        rows.append([int(w, 16) for w in line.split()])
    return rows


def test_philox_known_answers():
    rows = _kat_rows()
    assert len(rows) == 3
    for c0, c1, c2, c3, k0, k1, *expect in rows:
        got = philox.philox4x32_10(c0, c1, c2, c3, k0, k1)
        assert [int(w) for w in got] == expect


def test_philox_vectorised_matches_scalar():
    ctr = np.arange(50, dtype=np.uint64)
    vec = philox.philox4x32_10(ctr, 7, 3, 1, 11, 13)
    for i in (0, 17, 49):
        one = philox.philox4x32_10(i, 7, 3, 1, 11, 13)
        assert [int(v[i]) for v in vec] == [int(w) for w in one]


def test_seed_key_split():
    assert philox.seed_key(0x0123456789ABCDEF) == (0x89ABCDEF, 0x01234567)


def test_signs_are_rademacher():
    eps = rng.signs(1 << 16, seed=3, level=2)
    assert set(np.unique(eps)) == {-1, 1}
    n = eps.size
    assert abs(eps.astype(np.float64).mean()) < 5.0 / np.sqrt(n)
    # lag-1 correlation near zero (independent draws)
    e = eps.astype(np.float64)
    assert abs(np.mean(e[1:] * e[:-1])) < 5.0 / np.sqrt(n)
    # a different level gives a different vector
    assert np.mean(eps != rng.signs(1 << 16, seed=3, level=3)) > 0.45


def test_select_rows_brute_force():
    n_pad, m, seed, level = 256, 37, 11, 4
    keys = rng.row_keys(n_pad, seed, level)
    pairs = sorted((int(keys[i]), i) for i in range(n_pad))
    expect = sorted(i for _, i in pairs[:m])
    assert list(rng.select_rows(n_pad, m, seed, level)) == expect


def test_select_rows_structure():
    rows = rng.select_rows(4096, 300, seed=5, level=7)
    assert rows.size == 300 and np.all(np.diff(rows) > 0)
    assert rows.min() >= 0 and rows.max() < 4096
    assert list(rng.select_rows(64, 64, 1, 1)) == list(range(64))
    with pytest.raises(ValueError):
        rng.select_rows(64, 65, 1, 1)
    with pytest.raises(ValueError):
        rng.select_rows(64, 0, 1, 1)


def test_select_rows_uniform_inclusion():
    """Sampling without replacement, uniformly: each index is included with
    probability m / n_pad (chi-square over many seeds)."""
    n_pad, m, trials = 64, 8, 3000
    counts = np.zeros(n_pad)
    for s in range(trials):
        counts[rng.select_rows(n_pad, m, seed=s, level=0)] += 1
    expected = trials * m / n_pad
    chi2 = np.sum((counts - expected) ** 2 / expected)
    assert stats.chi2.sf(chi2, n_pad - 1) > 1e-4


def test_gaussian_distribution():
    z = rng.gaussian_z(64, 4096, seed=9, level=1).ravel()
    assert stats.kstest(z, "norm").pvalue > 1e-4
    assert abs(z.mean()) < 5 / np.sqrt(z.size)
    assert abs(z.var() - 1) < 0.03


def test_gaussian_rows_independent():
    z = rng.gaussian_z(8, 20000, seed=2, level=0)
    C = np.corrcoef(z)
    off = C[~np.eye(8, dtype=bool)]
    assert np.abs(off).max() < 5 / np.sqrt(20000)


def test_gaussian_column_blocks_consistent():
    full = rng.gaussian_z(10, 300, seed=4, level=3)
    part = rng.gaussian_z_cols(10, 100, 250, seed=4, level=3)
    assert np.array_equal(full[:, 100:250], part)
    # m that is not a multiple of four is a prefix of the next multiple
    assert np.array_equal(rng.gaussian_z(7, 50, 1, 1), rng.gaussian_z(8, 50, 1, 1)[:7])


def test_gaussian_uniforms_in_range():
    w = np.array([0, 1, 255, 256, 0xFFFFFFFF], dtype=np.uint64)
    u1 = rng._uniform_open0(w)
    u2 = rng._uniform_closed0(w)
    assert u1.min() > 0 and u1.max() == 1.0
    assert u2.min() == 0.0 and u2.max() < 1.0


def test_gaussian_rows_match_full():
    full = rng.gaussian_z(11, 200, seed=8, level=2)
    rows = [0, 3, 5, 10]
    assert np.array_equal(rng.gaussian_z_rows(rows, 200, seed=8, level=2), full[rows])


def test_sign_layout_known_answer():
    """Seed 0, level 0: block 0's first Philox call has key (0, 0) and counter
    (0, 0, 0, 0), whose output is the first published known answer.  Row
    q = 32 j + w (w < 4) of block 0 takes bit j of word w: eps = +1 for a 0 bit."""
    c0, c1, c2, c3, k0, k1, *words = _kat_rows()[0]
    assert (c0, c1, c2, c3, k0, k1) == (0, 0, 0, 0, 0, 0)
    eps = rng.signs(1024, seed=0, level=0)
    for w in range(4):
        for j in range(32):
            bit = (words[w] >> j) & 1
            assert eps[32 * j + w] == (1 if bit == 0 else -1), (w, j)


def test_sign_blocks_independent():
    """Every pair of 1024-row blocks is uncorrelated: a layout that reused one
    block's words for every block, or overlapped the counters of neighbouring
    blocks, gives correlations of 1 or about 1/2."""
    blocks = 64
    e = rng.signs(1024 * blocks, seed=1, level=2).astype(np.float64).reshape(blocks, 1024)
    corr = e @ e.T / 1024.0
    off = corr[~np.eye(blocks, dtype=bool)]
    assert np.max(np.abs(off)) < 5.0 / np.sqrt(1024.0)
    # and within a block the 32 words' bit columns are uncorrelated too
    w = e[0].reshape(32, 32)          # [bit j, word w] of block 0
    cw = w.T @ w / 32.0
    assert np.max(np.abs(cw[~np.eye(32, dtype=bool)])) < 0.8
