"""Pins of the oracle's linear algebra: closed-form solutions, the Woodbury
identity, Lemma 4.1 and the error recursion of App. B.1."""
import numpy as np
import pytest

from oracle import linalg, params, rng, sketch
from paper_2006_05874_gb300 import problems


def _svd_problem(n=200, d=12, seed=0):
    g = np.random.default_rng(seed)
    U, _ = np.linalg.qr(g.standard_normal((n, d)))
    V, _ = np.linalg.qr(g.standard_normal((d, d)))
    sigma = np.sort(g.uniform(0.05, 3.0, d))[::-1]
    A = (U * sigma) @ V.T
    b = g.standard_normal(n)
    return A, b, U, sigma, V


def test_direct_solve_matches_svd_closed_form():
    A, b, U, sigma, V = _svd_problem()
    nu = 0.3
    xs = linalg.direct_solve(A, b, nu)
    ref = linalg.svd_solve(U, sigma, V, b, nu)
    assert np.linalg.norm(xs - ref) <= 1e-12 * np.linalg.norm(ref)


def test_direct_solve_normal_equations_blocked():
    p = problems.exp_decay(n=3000, d=64, seed=1)
    A = p.A.astype(np.float64)
    xs = linalg.direct_solve(p.A, p.b, p.nu)
    res = A.T @ (A @ xs - p.b) + p.nu ** 2 * xs
    assert np.linalg.norm(res) <= 1e-10 * np.linalg.norm(A.T @ p.b.astype(np.float64))
    g_blk, ax2 = linalg.gradient_blocked(p.A, p.b, p.nu, xs, block=700)
    assert np.allclose(g_blk, linalg.gradient(p.A, p.b, p.nu, xs), atol=1e-9)
    assert np.isclose(ax2, np.sum((A @ xs) ** 2))


def test_gradient_is_derivative_of_objective():
    A, b, *_ = _svd_problem(n=50, d=6, seed=3)
    x = np.random.default_rng(4).standard_normal(6)
    nu, h = 0.7, 1e-6
    g = linalg.gradient(A, b, nu, x)
    fd = np.array([(linalg.objective(A, b, nu, x + h * e) - linalg.objective(A, b, nu, x - h * e)) / (2 * h)
                   for e in np.eye(6)])
    assert np.allclose(g, fd, rtol=1e-6, atol=1e-7)


def test_effective_dimension_definitions():
    A, b, U, sigma, V = _svd_problem(seed=5)
    nu = 0.4
    d = A.shape[1]
    explicit = np.trace(A @ np.linalg.solve(A.T @ A + nu ** 2 * np.eye(d), A.T))
    assert np.isclose(linalg.effective_dimension_trace(sigma, nu), explicit, rtol=1e-12)
    # ||D||_F^2 / ||D||_2^2 differs from the trace form by the factor ||D||_2^2 < 1
    D1 = sigma[0] ** 2 / (sigma[0] ** 2 + nu ** 2)
    assert np.isclose(linalg.effective_dimension_ratio(sigma, nu) * D1, explicit, rtol=1e-12)


def test_nu_for_target_hits_target():
    sigma = problems.poly_sigma(2048)
    nu = problems.nu_for_target(sigma, 100.0)
    assert abs(linalg.effective_dimension_trace(sigma, nu) - 100.0) < 1e-9
    assert abs(nu - 0.015313) < 5e-6


@pytest.mark.parametrize("m", [3, 12, 40])
def test_woodbury_matches_dense_solve(m):
    d = 12
    SA = problems.random_matrix(m, d, seed=m).astype(np.float64)
    g = np.random.default_rng(1).standard_normal(d)
    nu = 0.2
    F = linalg.WoodburyFactor(SA, nu)
    assert F.woodbury == (m < d)
    dense = np.linalg.solve(SA.T @ SA + nu ** 2 * np.eye(d), g)
    assert np.allclose(F.apply(g), dense, rtol=1e-10, atol=1e-12)


def _stack(A, nu):
    return np.vstack([A, nu * np.eye(A.shape[1])])


@pytest.mark.parametrize("kind", ["gauss", "srht"])
def test_lemma_4_1_decrement_identity(kind):
    """1/2 g^T H_S^{-1} g == 1/2 ||C_S^{-1/2} Ubar^T Abar (x - x*)||^2."""
    A, b, U, sigma, V = _svd_problem(n=128, d=10, seed=7)
    nu, m = 0.5, 24
    S = (rng.gaussian_embedding(m, 128, 1, 0) if kind == "gauss" else sketch.srht_matrix(128, m, 1, 0))
    x = np.random.default_rng(8).standard_normal(10)
    xs = linalg.direct_solve(A, b, nu)
    g = linalg.gradient(A, b, nu, x)
    r = linalg.newton_decrement(g, linalg.WoodburyFactor(S @ A, nu).apply(g))
    C = linalg.c_matrix(U, sigma, nu, S)
    e = linalg.ubar(U, sigma, V, nu).T @ _stack(A, nu) @ (x - xs)
    assert np.isclose(r, 0.5 * e @ np.linalg.solve(C, e), rtol=1e-9)


def test_c_matrix_is_ubar_sketch_gram():
    """C_S = Ubar^T Sbar^T Sbar Ubar with Sbar = blockdiag(S, I_d) (App. B.1)."""
    A, b, U, sigma, V = _svd_problem(n=64, d=5, seed=9)
    nu = 0.8
    S = rng.gaussian_embedding(20, 64, 2, 0)
    Ub = linalg.ubar(U, sigma, V, nu)
    assert np.allclose(Ub.T @ Ub, np.eye(5), atol=1e-12)
    Sbar = np.block([[S, np.zeros((20, 5))], [np.zeros((5, 64)), np.eye(5)]])
    assert np.allclose(linalg.c_matrix(U, sigma, nu, S), Ub.T @ Sbar.T @ Sbar @ Ub, atol=1e-10)


def test_gradient_ihs_error_recursion():
    """One gradient-IHS step maps e_t to (I - mu C_S^{-1}) e_t exactly (App. B.1),
    and one Polyak step follows the companion matrix M(mu, beta)."""
    A, b, U, sigma, V = _svd_problem(n=128, d=8, seed=11)
    nu, m = 0.3, 16
    S = sketch.srht_matrix(128, m, 4, 0)
    F = linalg.WoodburyFactor(S @ A, nu)
    xs = linalg.direct_solve(A, b, nu)
    Ub, Ab = linalg.ubar(U, sigma, V, nu), _stack(A, nu)
    C = linalg.c_matrix(U, sigma, nu, S)
    g = np.random.default_rng(12)
    x_prev, x = g.standard_normal(8), g.standard_normal(8)
    mu, beta = 0.7, 0.2
    x_gd = x - mu * F.apply(linalg.gradient(A, b, nu, x))
    e = lambda v: Ub.T @ Ab @ (v - xs)
    assert np.allclose(e(x_gd), (np.eye(8) - mu * np.linalg.inv(C)) @ e(x), atol=1e-10)
    x_p = x - mu * F.apply(linalg.gradient(A, b, nu, x)) + beta * (x - x_prev)
    Mtop = np.hstack([(1 + beta) * np.eye(8) - mu * np.linalg.inv(C), -beta * np.eye(8)])
    assert np.allclose(e(x_p), Mtop @ np.concatenate([e(x), e(x_prev)]), atol=1e-10)
    # delta_t = 1/2 ||e_t||^2
    assert np.isclose(0.5 * np.linalg.norm(e(x)) ** 2, 0.5 * np.linalg.norm(Ab @ (x - xs)) ** 2)


def test_theorem_2_1_contraction():
    """delta_{t+1} / delta_t <= c_gd(lambda, Lambda) with (lambda, Lambda) the
    extreme eigenvalues of C_S and mu = mu_gd(lambda, Lambda) (Thm 2.1)."""
    A, b, U, sigma, V = _svd_problem(n=256, d=10, seed=13)
    nu = 0.2
    S = rng.gaussian_embedding(60, 256, 5, 0)
    ev = np.linalg.eigvalsh(linalg.c_matrix(U, sigma, nu, S))
    lo, hi = ev[0], ev[-1]
    F = linalg.WoodburyFactor(S @ A, nu)
    xs = linalg.direct_solve(A, b, nu)
    Ab = _stack(A, nu)
    x = np.random.default_rng(14).standard_normal(10)
    for _ in range(5):
        x_new = x - params.mu_gd(lo, hi) * F.apply(linalg.gradient(A, b, nu, x))
        ratio = np.linalg.norm(Ab @ (x_new - xs)) ** 2 / np.linalg.norm(Ab @ (x - xs)) ** 2
        assert ratio <= params.c_gd(lo, hi) * (1 + 1e-9)
        x = x_new


def test_relative_error_metric():
    A, b, *_ = _svd_problem(n=40, d=4, seed=15)
    nu = 0.5
    xs = linalg.direct_solve(A, b, nu)
    assert linalg.relative_error(A, nu, xs, xs) == 0.0
    assert np.isclose(linalg.relative_error(A, nu, np.zeros(4), xs), 1.0)


def test_direct_solve_path_matches_single_points():
    """The shared-Gram path solve equals the closed form V diag(s/(s^2+nu^2)) U^T b
    at every nu (the path's A is built from known factors, in float64)."""
    g = np.random.default_rng(31)
    n, d = 600, 40
    U, _ = np.linalg.qr(g.standard_normal((n, d)))
    V, _ = np.linalg.qr(g.standard_normal((d, d)))
    s = np.arange(1, d + 1) ** -0.5
    A = (U * s) @ V.T
    nus = np.logspace(-3, 1, 5)
    bs = [g.standard_normal(n) for _ in nus]
    xs = linalg.direct_solve_path(A, bs, nus)
    for x, b, nu in zip(xs, bs, nus):
        ref = linalg.svd_solve(U, s, V, b, nu)
        assert np.linalg.norm(x - ref) <= 1e-10 * np.linalg.norm(ref)
