"""GPU CG and sketch-preconditioned CG (the Sec. 5 comparators) against the FP64
direct solution and the oracle's CG."""
import numpy as np
import pytest

from oracle import cg as oracle_cg
from oracle import linalg
from paper_2006_05874_gb300 import problems

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def spec_problem():
    p = problems.spectral(n=16384, d=256, de_target=30.0, seed=4)
    return p, linalg.direct_solve(p.A, p.b, p.nu)


def test_cg_reaches_direct_solution(ctx, torch_cuda, spec_problem):
    torch = torch_cuda
    p, xs = spec_problem
    x = torch.zeros(p.d, device="cuda")
    rep = ctx.cg(torch.from_numpy(p.A).cuda(), torch.from_numpy(p.b).cuda(), p.nu, x, tol=1e-8, max_iter=5000)
    assert rep.status == 0
    assert linalg.relative_error(p.A, p.nu, x.cpu().numpy(), xs) < 1e-5


def test_cg_iterations_match_oracle(ctx, torch_cuda, spec_problem):
    """Same algorithm, same stopping rule.  FP32 vectors lose the conjugacy of
    the search directions as the residual falls (kappa(H) ~ 400 here), which
    delays CG's superlinear phase: on this problem an FP32 CG needs 13 / 19
    iterations where the FP64 oracle needs 12 / 14 (tolerances 1e-3 / 1e-4).
    So the counts must agree at 1e-3 and may only grow, by at most half,
    at 1e-4."""
    torch = torch_cuda
    p, xs = spec_problem
    A, b = torch.from_numpy(p.A).cuda(), torch.from_numpy(p.b).cuda()
    x = torch.zeros(p.d, device="cuda")
    rep = ctx.cg(A, b, p.nu, x, tol=1e-3, max_iter=5000)
    _, it_ref, _ = oracle_cg.cg(p.A, p.b, p.nu, tol=1e-3, max_iter=5000)
    assert abs(rep.iterations - it_ref) <= 2
    x.zero_()
    rep = ctx.cg(A, b, p.nu, x, tol=1e-4, max_iter=5000)
    _, it_ref, _ = oracle_cg.cg(p.A, p.b, p.nu, tol=1e-4, max_iter=5000)
    assert it_ref - 1 <= rep.iterations <= 1.5 * it_ref + 2


@pytest.mark.parametrize("kind", ["srht", "gauss"])
def test_pcg_reaches_direct_solution(ctx, torch_cuda, spec_problem, kind):
    torch = torch_cuda
    p, xs = spec_problem
    x = torch.zeros(p.d, device="cuda")
    rep = ctx.cg(torch.from_numpy(p.A).cuda(), torch.from_numpy(p.b).cuda(), p.nu, x, tol=1e-8, max_iter=500,
                 precond=kind)
    assert rep.status == 0
    assert rep.m_final == oracle_cg.pcg_sketch_size(kind, p.n, p.d)
    assert linalg.relative_error(p.A, p.nu, x.cpu().numpy(), xs) < 1e-5
    assert rep.iterations < 30


def test_cg_rejects_bad_args(ctx, torch_cuda):
    from paper_2006_05874_gb300 import ihs

    torch = torch_cuda
    A = torch.zeros(8, 4, device="cuda")
    with pytest.raises(ihs.IHSError):
        ctx.cg(A, torch.zeros(8, device="cuda"), 0.0, torch.zeros(4, device="cuda"))
