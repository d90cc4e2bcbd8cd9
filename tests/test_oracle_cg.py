"""Pins of the CG / sketch-preconditioned CG comparators: convergence to the
direct solution, finite termination in exact arithmetic (at most d steps), a
one-step solve with the exact preconditioner, and the sketch sizes of Sec. 5."""
import math

import numpy as np

from oracle import cg, linalg
from paper_2006_05874_gb300 import problems


def test_cg_converges_to_direct_solution():
    p = problems.exp_decay(n=1024, d=64, seed=2)
    xs = linalg.direct_solve(p.A, p.b, p.nu)
    x, it, hist = cg.cg(p.A, p.b, p.nu, tol=1e-12, max_iter=5000)
    assert linalg.relative_error(p.A, p.nu, x, xs) < 1e-9
    assert hist[-1] <= 1e-12 * np.linalg.norm(p.A.astype(np.float64).T @ p.b)


def test_cg_terminates_within_d_steps_when_well_conditioned():
    g = np.random.default_rng(3)
    A = g.standard_normal((200, 12))
    b = g.standard_normal(200)
    x, it, _ = cg.cg(A, b, 1.0, tol=1e-13, max_iter=100)
    assert it <= 12 + 1
    assert np.allclose(x, linalg.direct_solve(A, b, 1.0), atol=1e-10)


def test_pcg_with_exact_preconditioner_is_one_step():
    g = np.random.default_rng(4)
    A = g.standard_normal((300, 20))
    b = g.standard_normal(300)
    nu = 0.3
    H = A.T @ A + nu * nu * np.eye(20)
    x, it, _ = cg.cg(A, b, nu, tol=1e-12, precond=lambda v: np.linalg.solve(H, v))
    assert it == 1


def test_pcg_sketch_sizes():
    assert cg.pcg_sketch_size("gauss", 10 ** 6, 2048, 0.1) == 20480
    assert cg.pcg_sketch_size("srht", 10 ** 6, 256, 0.1) == math.ceil(256 * math.log(256) / 0.1)
    assert cg.pcg_sketch_size("srht", 131072, 2048, 0.1) == 131072   # capped at n_pad


def test_pcg_converges_fast():
    p = problems.exp_decay(n=4096, d=64, seed=5)
    xs = linalg.direct_solve(p.A, p.b, p.nu)
    x, it, hist, m = cg.pcg(p.A, p.b, p.nu, kind="gauss", tol=1e-10)
    x_cg, it_cg, _ = cg.cg(p.A, p.b, p.nu, tol=1e-10, max_iter=10000)
    assert linalg.relative_error(p.A, p.nu, x, xs) < 1e-7
    assert it < it_cg
