"""Pins of the oracle's dual (underdetermined, App. A.2) mode against closed forms:
the dual optimum (A A^T + nu^2 I) z* = b, the primal-dual map x* = A^T z*, and the
push-through identity A^T (A A^T + nu^2 I)^-1 b = (A^T A + nu^2 I)^-1 A^T b."""
import numpy as np
import pytest

from oracle import ihs, linalg


def _problem(n, d, seed, decay=0.995):
    rng = np.random.default_rng(seed)
    A = rng.standard_normal((n, d)) * (decay ** np.arange(d))[None, :] / np.sqrt(d)
    b = rng.standard_normal(n)
    return A, b


@pytest.mark.parametrize("kind", ["srht", "gauss"])
def test_dual_converges_to_primal_direct_solution(kind):
    A, b = _problem(48, 700, seed=1)
    nu = 0.05
    x, res = ihs.adaptive_ihs_dual(A, b, nu, kind=kind, tol=1e-11, seed=3)
    assert res.status == "converged"
    xs = linalg.direct_solve(A, b, nu)
    assert np.linalg.norm(A @ (x - xs)) / np.linalg.norm(A @ xs) <= 1e-8
    assert np.linalg.norm(x - xs) / np.linalg.norm(xs) <= 1e-7


def test_dual_optimum_closed_form():
    A, b = _problem(32, 300, seed=2)
    nu = 0.2
    x, res = ihs.adaptive_ihs_dual(A, b, nu, tol=1e-12)
    z_star = np.linalg.solve(A @ A.T + nu * nu * np.eye(A.shape[0]), b)
    assert np.allclose(res.x, z_star, rtol=1e-8, atol=1e-10 * np.abs(z_star).max())
    # the dual gradient A A^T z - b + nu^2 z vanishes there, the one without nu^2 z does not
    assert np.linalg.norm(A @ (A.T @ z_star) - b + nu * nu * z_star) <= 1e-10 * np.linalg.norm(b)
    assert np.linalg.norm(A @ (A.T @ z_star) - b) > 1e-3 * np.linalg.norm(b)


def test_push_through_identity():
    A, b = _problem(20, 90, seed=4)
    nu = 0.7
    lhs = A.T @ np.linalg.solve(A @ A.T + nu * nu * np.eye(20), b)
    rhs = np.linalg.solve(A.T @ A + nu * nu * np.eye(90), A.T @ b)
    assert np.allclose(lhs, rhs, rtol=1e-10, atol=1e-12)
    assert np.allclose(lhs, linalg.direct_solve(A, b, nu), rtol=1e-10, atol=1e-12)
    assert np.allclose(linalg.direct_solve_dual(A, b, nu), rhs, rtol=1e-10, atol=1e-12)


def test_dual_levels_keyed_like_the_primal():
    # the dual runs the same controller on A^T: a warm start at m = 2^l replays
    # the cold run's draws from level l on, so it ends at the same level
    A, b = _problem(40, 600, seed=5)
    nu = 0.05
    _, cold = ihs.adaptive_ihs_dual(A, b, nu, tol=1e-9)
    m0 = cold.levels[-1]
    _, warm = ihs.adaptive_ihs_dual(A, b, nu, tol=1e-9, m_init=m0)
    assert warm.levels[0] == m0 and warm.levels[-1] == m0
    assert warm.status == "converged"
