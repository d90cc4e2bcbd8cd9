"""Pins of the parameter formulas (closed forms of Thm 2.1/2.2, Def 3.1/3.2,
Lemma B.1, Lemma B.2) and of the adaptive method (convergence to the direct
solution, the acceptance invariants, the rate bound of the proofs of
Thm 4.1/4.2, the sketch-size bound of Thm 4.1)."""
import math

import numpy as np
import pytest

from oracle import hadamard, ihs, linalg, params, rng, sketch
from paper_2006_05874_gb300 import problems


def test_srht_parameters_closed_form():
    """Def 3.2: mu_gd = 1 - rho and c_gd = rho (App. B.3 states c_gd(rho) = rho)."""
    for rho in (0.01, 0.1, 0.3, 0.7):
        p = params.ihs_params("srht", rho)
        assert math.isclose(p.mu_gd, 1 - rho, rel_tol=1e-14)
        assert math.isclose(p.c_gd, rho, rel_tol=1e-13)
        assert p.beta_p == p.c_p


def test_gaussian_parameters_closed_form():
    """Def 3.1 with s^2 = c_eta rho: beta_p = c_p = s^2, mu_p = (1 - s^2)^2,
    c_gd = (2 s / (1 + s^2))^2, mu_gd = (1 - s^2)^2 / (1 + s^2)."""
    for rho, eta in ((0.1, 0.01), (0.05, 0.001), (0.18, 0.01)):
        s2 = (1 + 3 * math.sqrt(eta)) ** 2 * rho
        p = params.ihs_params("gauss", rho, eta)
        assert math.isclose(p.beta_p, s2, rel_tol=1e-12)
        assert math.isclose(p.mu_p, (1 - s2) ** 2, rel_tol=1e-12)
        assert math.isclose(p.c_gd, (2 * math.sqrt(s2) / (1 + s2)) ** 2, rel_tol=1e-12)
        assert math.isclose(p.mu_gd, (1 - s2) ** 2 / (1 + s2), rel_tol=1e-12)


def test_parameter_values_default():
    g = params.ihs_params("gauss", 0.1, 0.01)
    assert abs(g.mu_gd - 0.59073) < 1e-4 and abs(g.c_gd - 0.49467) < 1e-4
    assert abs(g.mu_p - 0.69056) < 1e-4 and abs(g.beta_p - 0.169) < 1e-9
    s = params.ihs_params("srht", 0.1)
    assert abs(s.mu_p - 0.92370) < 1e-4 and abs(s.beta_p - 0.026334) < 1e-5


def test_parameter_domain_checks():
    with pytest.raises(ValueError):
        params.bounds_gaussian(0.2, 0.01)
    with pytest.raises(ValueError):
        params.bounds_srht(1.0)


def test_lemma_b1_gaussian_ratio():
    """On E_{rho/5}: (Lambda/lambda)(rho/5) * c_gd(rho/5) <= c_gd(rho) (Lemma B.1)."""
    for rho in np.linspace(0.01, 0.18, 12):
        lo5, hi5 = params.bounds_gaussian(rho / 5, 0.01)
        lo, hi = params.bounds_gaussian(rho, 0.01)
        assert hi5 / lo5 * params.c_gd(lo5, hi5) <= params.c_gd(lo, hi)


def test_lemma_b2_srht_ratio():
    """a_rho = (1+sqrt rho)/(1-sqrt rho) bounds the spread on E_{rho/a} and
    c_gd(rho/a) = c_gd(rho)/a (Lemma B.2)."""
    for rho in (0.05, 0.1, 0.5):
        a = (1 + math.sqrt(rho)) / (1 - math.sqrt(rho))
        lo, hi = params.bounds_srht(rho / a)
        assert hi / lo < a
        assert math.isclose(params.c_gd(lo, hi), params.c_gd(*params.bounds_srht(rho)) / a, rel_tol=1e-12)


def test_polyak_rate_theorem_2_2():
    """With (mu_p, beta_p), every 2x2 block M_i of App. B.1 has spectral radius
    sqrt(beta_p) for any gamma_i in [lambda, Lambda] (Thm 2.2)."""
    lo, hi = 0.4, 2.5
    mu, beta = params.mu_p(lo, hi), params.beta_p(lo, hi)
    for gam in np.linspace(lo, hi, 9):
        M = np.array([[1 + beta - mu / gam, -beta], [1, 0]])
        assert np.abs(np.linalg.eigvals(M)).max() <= math.sqrt(beta) * (1 + 1e-7)


@pytest.fixture(scope="module")
def exp_problem():
    p = problems.exp_decay(n=2048, d=128, seed=0)
    xs = linalg.direct_solve(p.A, p.b, p.nu)
    return p, xs


@pytest.mark.parametrize("kind", ["srht", "gauss"])
@pytest.mark.parametrize("variant", ["gd", "polyak"])
def test_adaptive_ihs_reaches_direct_solution(exp_problem, kind, variant):
    p, xs = exp_problem
    res = ihs.adaptive_ihs(p.A, p.b, p.nu, kind=kind, variant=variant, tol=1e-6)
    assert res.status == "converged"
    assert linalg.relative_error(p.A, p.nu, res.x, xs) < 1e-6
    prm = params.ihs_params(kind)
    # acceptance invariants of the two candidates
    for ev, t, m, ratio in res.trace:
        if ev == "gd":
            assert ratio <= prm.c_gd
        elif ev == "polyak":
            assert ratio <= prm.c_p
        elif ev == "polyak_reject":
            assert ratio > prm.c_p
        elif ev == "stop":
            assert ratio <= 1.0
        elif ev == "double":
            assert ratio > prm.c_gd
    # the schedule is a doubling sequence
    assert all(b == 2 * a for a, b in zip(res.levels, res.levels[1:]))


def test_adaptive_ihs_rate_bound_srht():
    """r_t / r_1 <= c_gd^(t-1) by construction, hence
    delta_t / delta_1 <= sigma_max(C_S) / sigma_min(C_S_init) c_gd^(t-1) with
    sigma_min(C_S_init) >= nu^2/(sigma_1^2 + nu^2) (proof of Thm 4.2)."""
    g = np.random.default_rng(21)
    n, d = 256, 16
    U, _ = np.linalg.qr(g.standard_normal((n, d)))
    V, _ = np.linalg.qr(g.standard_normal((d, d)))
    sigma = 0.8 ** np.arange(d) * 4
    A = (U * sigma) @ V.T
    b = A @ g.standard_normal(d) + 0.1 * g.standard_normal(n)
    nu = 0.05
    xs = linalg.direct_solve(A, b, nu)
    res = ihs.adaptive_ihs(A, b, nu, kind="srht", variant="gd", tol=1e-9, keep_history=True)
    Ab = np.vstack([A, nu * np.eye(d)])
    delta = lambda x: 0.5 * np.linalg.norm(Ab @ (x - xs)) ** 2
    d1 = delta(res.history[0][1])
    c = params.ihs_params("srht").c_gd
    for t, x, SA in res.history:
        # sigma_max(C_S) through the Rayleigh quotient of H_S against H
        H = A.T @ A + nu ** 2 * np.eye(d)
        HS = SA.T @ SA + nu ** 2 * np.eye(d)
        smax = np.linalg.eigvalsh(np.linalg.solve(np.linalg.cholesky(H), np.linalg.solve(np.linalg.cholesky(H), HS).T)).max()
        bound = smax * (1 + sigma[0] ** 2 / nu ** 2) * c ** (t - 1)
        assert delta(x) / d1 <= bound * (1 + 1e-9)


def test_sketch_size_bound_gaussian():
    """Settled m <= 2 c0 d_e / rho with c0 = 5 (Thm 4.1; w.h.p.)."""
    p = problems.spectral(n=4096, d=256, sigma=0.7 ** np.arange(256), de_target=6.0, seed=3)
    de = linalg.effective_dimension_ratio(p.sigma, p.nu)
    res = ihs.adaptive_ihs(p.A, p.b, p.nu, kind="gauss", variant="gd", tol=1e-8)
    assert res.status == "converged"
    assert res.m <= params.sketch_size_bound("gauss", de, 0.1)
    assert len(res.levels) - 1 <= params.rejected_steps_bound("gauss", de, 0.1) + 1e-9


def test_srht_at_cap_is_exact_newton():
    """m = n_pad: S is orthogonal, H_S = H, one gradient step of size 1 solves
    the problem, so gt_1 = H^{-1} g_1 = x_1 - x*."""
    p = problems.exp_decay(n=64, d=8, seed=4)
    xs = linalg.direct_solve(p.A, p.b, p.nu)
    SA = sketch.srht_sketch(p.A, 64, seed=0, level=6)
    F = linalg.WoodburyFactor(SA, p.nu)
    x1 = np.zeros(8)
    gt = F.apply(linalg.gradient(p.A, p.b, p.nu, x1))
    assert np.allclose(x1 - gt, xs, rtol=1e-9, atol=1e-9)


def test_warm_start_level_reuses_draws():
    """Sketches are keyed by (seed, level): starting at m = 2^l replays the
    level-l draws of a run started at m = 1."""
    p = problems.exp_decay(n=512, d=32, seed=5)
    cold = ihs.adaptive_ihs(p.A, p.b, p.nu, kind="srht", tol=1e-8)
    m_last = cold.levels[-1]
    warm = ihs.adaptive_ihs(p.A, p.b, p.nu, kind="srht", tol=1e-8, m_init=m_last)
    assert warm.levels == [m_last]
    assert warm.status == "converged"


def test_floor_guard_stops_instead_of_doubling():
    p = problems.exp_decay(n=4096, d=32, seed=6)
    res = ihs.adaptive_ihs(p.A, p.b, p.nu, kind="srht", tol=0.0, floor=1e-3, max_iter=500)
    assert res.status == "floor"
    assert res.r <= 1e-6 * res.r1 and res.trace[-1][0] == "floor"
