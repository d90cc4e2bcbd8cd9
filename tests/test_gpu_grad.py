"""Parity of the fused gradient pass g = A^T(Ax - b) + nu^2 x with the FP64 oracle.

Tolerance (derived from the arithmetic): the kernel forms r_i with a Dot2
(compensated) dot product and accumulates A^T r with compensated sums, so the
dominant error is rounding r_i and g_c to binary32 (relative u = 2^-24 each):
|dg_c| <= 2u |g_c| + 16u ||(r_i a_ic)_i||_2 + 16u nu^2 |x_c|
(random rounding errors add up like a random walk; 16 is a safety factor).
"""
import numpy as np
import pytest

from oracle import linalg
from paper_2006_05874_gb300 import problems

pytestmark = pytest.mark.gpu
U = 2.0 ** -24


def _check(torch, ctx, A, b, nu, x):
    Ag, bg, xg = (torch.from_numpy(np.ascontiguousarray(v)).cuda() for v in (A, b, x))
    g = torch.empty(A.shape[1], dtype=torch.float32, device="cuda")
    ax2 = ctx.grad(Ag, bg, nu, xg, g)
    g = g.cpu().numpy().astype(np.float64)
    A64, b64, x64 = A.astype(np.float64), b.astype(np.float64), x.astype(np.float64)
    Ax = A64 @ x64
    r = Ax - b64
    g_ref = A64.T @ r + nu * nu * x64
    scale = np.sqrt((r[:, None] ** 2 * A64 ** 2).sum(axis=0))
    tol = 2 * U * np.abs(g_ref) + 16 * U * scale + 16 * U * nu * nu * np.abs(x64) + 1e-30
    err = np.abs(g - g_ref)
    assert np.all(err <= tol), (err / tol).max()
    assert abs(ax2 - Ax @ Ax) <= 1e-6 * (Ax @ Ax) + 1e-30
    return g


@pytest.mark.parametrize("n,d", [(1, 4), (7, 8), (1000, 32), (4096, 128), (4099, 256), (3000, 512),
                                 (2500, 1024), (1000, 2048), (700, 4096), (300, 8192),
                                 (1001, 2048), (333, 1056), (5, 2048), (701, 4096), (3, 8192),
                                 (100, 37), (513, 3), (50, 9000)])
def test_grad_random_point(ctx, torch_cuda, n, d):
    A = problems.random_matrix(n, d, seed=n + d)
    b = problems.random_vector(n, seed=n)
    x = problems.random_vector(d, seed=d)
    _check(torch_cuda, ctx, A, b, 0.3, x)


def test_grad_near_solution_exp_decay(ctx, torch_cuda):
    """At x ~ x* the gradient cancels heavily; the compensated sums keep it."""
    p = problems.exp_decay(n=4096, d=256, seed=0)
    xs = linalg.direct_solve(p.A, p.b, p.nu).astype(np.float32)
    g = _check(torch_cuda, ctx, p.A, p.b, p.nu, xs)
    assert np.linalg.norm(g) < 1e-3 * np.linalg.norm(p.A.astype(np.float64).T @ p.b)


@pytest.mark.parametrize("d", [512, 2048])
def test_grad_deterministic(ctx, torch_cuda, d):
    torch = torch_cuda
    A = torch.from_numpy(problems.random_matrix(20000, d, seed=1)).cuda()
    b = torch.from_numpy(problems.random_vector(20000, seed=2)).cuda()
    x = torch.from_numpy(problems.random_vector(d, seed=3)).cuda()
    outs = []
    for _ in range(3):
        g = torch.empty(d, device="cuda")
        ctx.grad(A, b, 0.1, x, g)
        outs.append(g.cpu().numpy())
    assert all(np.array_equal(outs[0], o) for o in outs[1:])


def test_grad_full_size_spectral_shape(ctx, torch_cuda):
    """131072 x 2048 (the measured workload's shape), checked component-wise."""
    A = problems.random_matrix(131072, 2048, seed=5, scale=1.0 / 45.0)
    b = problems.random_vector(131072, seed=6, scale=0.01)
    x = problems.random_vector(2048, seed=7)
    _check(torch_cuda, ctx, A, b, 0.015, x)


def test_grad_rejects_bad_args(ctx, torch_cuda):
    from paper_2006_05874_gb300 import ihs

    torch = torch_cuda
    A = torch.zeros(4, 4, device="cuda")
    v = torch.zeros(4, device="cuda")
    with pytest.raises(ihs.IHSError):
        ctx.grad(A, v, -1.0, v, v)
