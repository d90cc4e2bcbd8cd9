"""Pins of the nested ("incremental") sketches: with every level keyed like
level 0, the Gaussian S_2m A starts with sqrt(1/2) S_m A, the SRHT rows of size m
are a subset of those of size 2m with the same signs, and the adaptive method on
nested draws still converges to the direct solution."""
import numpy as np
import pytest

from oracle import ihs, linalg, rng, sketch
from paper_2006_05874_gb300 import problems


def test_gaussian_prefix_property():
    A = problems.random_matrix(700, 30, seed=1).astype(np.float64)
    for m in (1, 4, 16):
        small = sketch.gaussian_sketch(A, m, 9, 0)
        big = sketch.gaussian_sketch(A, 2 * m, 9, 0)
        assert np.allclose(big[:m] * np.sqrt(2.0), small, rtol=1e-13, atol=1e-13)
    # a level-keyed draw is not nested
    assert not np.allclose(sketch.gaussian_sketch(A, 8, 9, 4)[:4] * np.sqrt(2.0), sketch.gaussian_sketch(A, 4, 9, 3))


def test_srht_rows_nested():
    n_pad = 4096
    prev = set()
    for m in (1, 2, 4, 64, 1024):
        rows = set(rng.select_rows(n_pad, m, 5, 0).tolist())
        assert prev <= rows and len(rows) == m
        prev = rows
    # the same signs at every size: S_m A is a row subset of S_2m A up to sqrt(2)
    A = problems.random_matrix(3000, 12, seed=2).astype(np.float64)
    s8, s16 = sketch.srht_sketch(A, 8, 5, 0), sketch.srht_sketch(A, 16, 5, 0)
    r8, r16 = rng.select_rows(4096, 8, 5, 0), list(rng.select_rows(4096, 16, 5, 0))
    for k, r in enumerate(r8):
        assert np.allclose(s16[r16.index(r)] * np.sqrt(2.0), s8[k], rtol=1e-12, atol=1e-12)


@pytest.mark.parametrize("kind", ["srht", "gauss"])
def test_nested_run_converges(kind):
    p = problems.exp_decay(2048, 64, seed=3)
    res = ihs.adaptive_ihs(p.A, p.b, p.nu, kind=kind, tol=1e-9, nested=True)
    assert res.status == "converged"
    xs = linalg.direct_solve(p.A, p.b, p.nu)
    assert linalg.relative_error(p.A, p.nu, res.x, xs) <= 1e-8
