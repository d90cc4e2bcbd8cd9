"""The synthetic input recipes (CPU): the spectra and effective dimensions they
promise, and their determinism in the seed."""
import math

import numpy as np
import pytest

from paper_2006_05874_gb300 import problems


def _de(sigma, nu):
    return float(np.sum(sigma ** 2 / (sigma ** 2 + nu * nu)))


def test_spectral_has_its_singular_values_and_target():
    p = problems.spectral(n=1024, d=48, de_target=12.0, seed=3)
    s = np.linalg.svd(p.A.astype(np.float64), compute_uv=False)
    assert np.allclose(s, p.sigma, rtol=1e-5, atol=1e-7)       # Haar U, V: exactly sigma (FP32 rounding)
    assert _de(p.sigma, p.nu) == pytest.approx(12.0, rel=1e-9)
    r = p.b.astype(np.float64) - p.A.astype(np.float64) @ p.x0
    assert np.std(r) == pytest.approx(0.01, rel=0.15)            # b = A x0 + 0.01 N(0, I)


def test_spectral_is_seeded():
    a = problems.spectral(n=256, d=16, de_target=4.0, seed=5)
    b = problems.spectral(n=256, d=16, de_target=4.0, seed=5)
    c = problems.spectral(n=256, d=16, de_target=4.0, seed=6)
    assert np.array_equal(a.A, b.A) and np.array_equal(a.b, b.b)
    assert not np.array_equal(a.A, c.A)


def test_exp_decay_columns_scale():
    p = problems.exp_decay(n=20000, d=32, seed=1)
    norms = np.linalg.norm(p.A.astype(np.float64), axis=0) / math.sqrt(20000)
    want = 0.95 ** np.arange(1, 33)
    assert np.allclose(norms, want, rtol=0.03)                   # a_ij ~ N(0, 1) 0.95^j
    assert p.nu == 0.1


def test_nu_for_target_monotone():
    sigma = problems.poly_sigma(500, 1.0)
    nus = [problems.nu_for_target(sigma, t) for t in (5.0, 20.0, 100.0)]
    assert nus[0] > nus[1] > nus[2] > 0
    for t, nu in zip((5.0, 20.0, 100.0), nus):
        assert _de(sigma, nu) == pytest.approx(t, rel=1e-9)
