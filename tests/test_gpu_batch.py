"""Batched solves (ihs_solve_batched): every problem of a batch against the FP64
oracle's direct solution at the single solver's bar (1e-5 relative prediction
norm), the schedule against the single solver's, and the edge cases."""
import math

import numpy as np
import pytest

from oracle import linalg
from paper_2006_05874_gb300 import problems

pytestmark = pytest.mark.gpu


def _dev(torch, a):
    return torch.as_tensor(np.ascontiguousarray(a, dtype=np.float32), device="cuda")


def _independent(seed, count, nmax=4096, dmax=256):
    """Gaussian-entry problems with n >= 16 d (a Gaussian sketch needs room to
    grow to about d_e / rho rows below its cap m = n)."""
    rng = np.random.default_rng(seed)
    out = []
    for i in range(count):
        d = int(rng.integers(8, dmax + 1))
        n = int(rng.integers(16 * d, max(16 * d, nmax) + 1))
        A = rng.standard_normal((n, d)).astype(np.float32)
        x0 = rng.standard_normal(d)
        b = (A @ x0 + 0.1 * rng.standard_normal(n)).astype(np.float32)
        out.append((A, b, 1.0))
    return out


def _path(n=8192, d=256, K=8, seed=3):
    rng = np.random.default_rng(seed)
    p = problems.spectral(n, d, sigma=np.arange(1, d + 1) ** -0.5, nu=0.1, seed=seed)
    nus = np.logspace(-3, 1, K)
    bs = []
    for k in range(K):
        x0 = rng.standard_normal(d)
        bs.append((p.A.astype(np.float64) @ x0 + 0.01 * rng.standard_normal(n)).astype(np.float32))
    return p.A, bs, nus


@pytest.mark.parametrize("kind", ["srht", "gauss"])
def test_batch_independent_matches_oracle_and_single(ctx, torch_cuda, kind):
    torch = torch_cuda
    ctx.set_params(kind=kind, variant="gd")
    probs = _independent(11, 7, nmax=4096, dmax=128)
    dev = [(_dev(torch, A), _dev(torch, b), nu, torch.zeros(A.shape[1], device="cuda")) for A, b, nu in probs]
    reps = ctx.solve_batched(dev)
    for (A, b, nu), (Ad, bd, _, x), rep in zip(probs, dev, reps):
        assert rep.status == 0
        xs = linalg.direct_solve(A, b, nu)
        assert linalg.relative_error(A, nu, x.cpu().numpy(), xs) <= 1e-5
        # the single solver on the same problem takes the same schedule
        x1 = torch.zeros(A.shape[1], device="cuda")
        r1 = ctx.solve(Ad, bd, nu, x1)
        assert rep.levels() == r1.levels()
        assert rep.iterations == r1.iterations


def test_batch_ridge_path_shared_A(ctx, torch_cuda):
    torch = torch_cuda
    ctx.set_params(kind="srht", variant="gd")
    A, bs, nus = _path()
    Ad = _dev(torch, A)
    dev = [(Ad, _dev(torch, b), nu, torch.zeros(A.shape[1], device="cuda")) for b, nu in zip(bs, nus)]
    reps = ctx.solve_batched(dev)
    for b, nu, (_, _, _, x), rep in zip(bs, nus, dev, reps):
        assert rep.status == 0
        xs = linalg.direct_solve(A, b, nu)
        assert linalg.relative_error(A, nu, x.cpu().numpy(), xs) <= 1e-5, nu
    # larger nu: smaller effective dimension, the doubling stops earlier
    assert reps[-1].m_final <= reps[0].m_final


def test_batch_mixed_groups_and_singletons(ctx, torch_cuda):
    torch = torch_cuda
    ctx.set_params(kind="gauss", variant="gd")
    A, bs, nus = _path(n=4096, d=128, K=3, seed=5)
    Ad = _dev(torch, A)
    dev = [(Ad, _dev(torch, b), nu, torch.zeros(A.shape[1], device="cuda")) for b, nu in zip(bs, nus)]
    ind = _independent(12, 3, nmax=3000, dmax=96)
    dev += [(_dev(torch, a), _dev(torch, b), nu, torch.zeros(a.shape[1], device="cuda")) for a, b, nu in ind]
    host = [(A, b, nu) for b, nu in zip(bs, nus)] + ind
    reps = ctx.solve_batched(dev)
    for (Ah, b, nu), (_, _, _, x), rep in zip(host, dev, reps):
        assert rep.status == 0
        assert linalg.relative_error(Ah, nu, x.cpu().numpy(), linalg.direct_solve(Ah, b, nu)) <= 1e-5


def test_batch_edge_cases(ctx, torch_cuda):
    torch = torch_cuda
    ctx.set_params(kind="srht", variant="gd")
    rng = np.random.default_rng(7)
    A = rng.standard_normal((500, 20)).astype(np.float32)
    b0 = np.zeros(500, dtype=np.float32)                      # x = 0 is the solution
    b1 = (A @ rng.standard_normal(20)).astype(np.float32)
    dev = [(_dev(torch, A), _dev(torch, b0), 0.5, torch.zeros(20, device="cuda")),
           (_dev(torch, A.copy()), _dev(torch, b1), 0.5, torch.zeros(20, device="cuda"))]
    reps = ctx.solve_batched(dev)
    assert reps[0].status == 0 and reps[0].iterations == 1
    assert np.all(dev[0][3].cpu().numpy() == 0.0)
    assert linalg.relative_error(A, 0.5, dev[1][3].cpu().numpy(), linalg.direct_solve(A, b1, 0.5)) <= 1e-5
    # a single problem in a batch
    x = torch.zeros(20, device="cuda")
    rep = ctx.solve_batched([(dev[1][0], dev[1][1], 0.5, x)])[0]
    assert rep.status == 0
    # iteration limit reported per problem
    ctx.set_params(max_iter=2)
    x = torch.zeros(20, device="cuda")
    rep = ctx.solve_batched([(dev[1][0], dev[1][1], 1e-3, x)])[0]
    assert rep.status == -6 and rep.iterations == 2
    ctx.set_params(max_iter=1000)


def test_batch_rejects_polyak_and_bad_args(ctx, torch_cuda):
    from paper_2006_05874_gb300 import ihs

    torch = torch_cuda
    A = torch.zeros(16, 4, device="cuda")
    b = torch.zeros(16, device="cuda")
    x = torch.zeros(4, device="cuda")
    ctx.set_params(variant="polyak")
    with pytest.raises(ihs.IHSError):
        ctx.solve_batched([(A, b, 1.0, x)])
    ctx.set_params(variant="gd")
    with pytest.raises(ihs.IHSError):
        ctx.solve_batched([(A, b, -1.0, x)])


def test_batch_per_problem_initial_sizes(ctx, torch_cuda):
    """m_init per problem (as a warm start supplies it): same accuracy, and the
    schedule starts at the given size."""
    torch = torch_cuda
    ctx.set_params(kind="srht", variant="gd")
    probs = _independent(21, 4, nmax=4096, dmax=128)
    dev = [(_dev(torch, A), _dev(torch, b), nu, torch.zeros(A.shape[1], device="cuda")) for A, b, nu in probs]
    m0 = [64, 128, 1, 256]
    reps = ctx.solve_batched(dev, m_init=m0)
    for (A, b, nu), (_, _, _, x), rep, m in zip(probs, dev, reps, m0):
        assert rep.status == 0
        assert rep.levels()[0] == m
        assert linalg.relative_error(A, nu, x.cpu().numpy(), linalg.direct_solve(A, b, nu)) <= 1e-5
    with pytest.raises(Exception):
        ctx.solve_batched(dev[:1], m_init=[3])


def test_batch_config4_scale_sample(ctx, torch_cuda):
    """At the batched workload's own scale: a 32-point ridge path on one
    262144 x 1024 A (sigma_j = j^-1/2, nu log-spaced over the workload's
    1e-4 .. 1e1, every other point of its 64) plus 32 independent Gaussian-entry
    problems from its recipe (n ~ U{2^10..2^14}, d ~ U{32..512}, nu = 1), in one
    batch; every one of the 64 solutions against the FP64 direct solve."""
    torch = torch_cuda
    ctx.set_params(kind="srht", variant="gd", tol=1e-5, m_init=1, max_iter=1000)
    n, d = 262144, 1024
    p = problems.spectral(n, d, sigma=np.arange(1, d + 1) ** -0.5, nu=1.0, seed=41, device="cuda")
    nus = np.logspace(-4, 1, 64)[::2]
    rng = np.random.default_rng(41)
    A64 = p.A.astype(np.float64)
    bs = [(A64 @ rng.standard_normal(d) + 0.01 * rng.standard_normal(n)).astype(np.float32) for _ in nus]
    ind = []
    for _ in range(32):
        nn = int(rng.integers(1 << 10, (1 << 14) + 1))
        dd = int(rng.integers(32, 513))
        A = rng.standard_normal((nn, dd)).astype(np.float32)
        b = (A @ rng.standard_normal(dd) + 0.1 * rng.standard_normal(nn)).astype(np.float32)
        ind.append((A, b, 1.0))
    Ad = _dev(torch, p.A)
    dev = [(Ad, _dev(torch, b), float(nu), torch.zeros(d, device="cuda")) for b, nu in zip(bs, nus)]
    dev += [(_dev(torch, A), _dev(torch, b), nu, torch.zeros(A.shape[1], device="cuda")) for A, b, nu in ind]
    reps = ctx.solve_batched(dev)
    xs_path = linalg.direct_solve_path(p.A, bs, nus)
    worst = 0.0
    for k, (xs, nu) in enumerate(zip(xs_path, nus)):
        assert reps[k].status == 0, (k, reps[k].status)
        err = linalg.relative_error(p.A, nu, dev[k][3].cpu().numpy(), xs)
        worst = max(worst, err)
        assert err <= 1e-5, (nu, err)
    for k, (A, b, nu) in enumerate(ind):
        rep = reps[len(nus) + k]
        assert rep.status == 0
        err = linalg.relative_error(A, nu, dev[len(nus) + k][3].cpu().numpy(), linalg.direct_solve(A, b, nu))
        worst = max(worst, err)
        assert err <= 1e-5, (A.shape, err)
