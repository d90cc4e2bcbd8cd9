"""The underdetermined case (App. A.2) on the GPU against the FP64 oracle's dual
run: the primal solution x = A^T z within 1e-5 relative prediction-norm error of
the direct solution, and the dual doubling schedule equal to the oracle's."""
import numpy as np
import pytest

from oracle import ihs as oracle_ihs
from oracle import linalg
from paper_2006_05874_gb300 import problems
from schedule_parity import assert_same_schedule

pytestmark = pytest.mark.gpu
# The dual's own stopping criterion; the primal error is up to sigma_1^2 / nu^2
# times larger (App. A.2), so each case takes the tolerance at which the
# oracle's dual run meets 1e-5 on x (exp. decay: sigma_1^2 / nu^2 = 3.7e5).


def _run(ctx, torch, A, b, nu, kind, tol):
    ctx.set_params(kind=kind, variant="gd", tol=tol, m_init=1)
    x = torch.full((A.shape[1],), float("nan"), device="cuda")
    rep = ctx.solve_dual(torch.from_numpy(np.ascontiguousarray(A, dtype=np.float32)).cuda(),
                         torch.from_numpy(np.ascontiguousarray(b, dtype=np.float32)).cuda(), nu, x)
    return rep, x.cpu().numpy().astype(np.float64)


@pytest.mark.parametrize("kind", ["srht", "gauss"])
def test_dual_exp_decay(ctx, torch_cuda, kind):
    p = problems.exp_decay(n=4096, d=256, seed=0)
    A = np.ascontiguousarray(p.A.T)                       # 256 x 4096: n < d
    b = np.random.default_rng(1).standard_normal(A.shape[0]).astype(np.float32)
    A64 = A.astype(np.float64)
    rep, x = _run(ctx, torch_cuda, A, b, p.nu, kind, 1e-8)
    assert rep.status == 0
    xs = linalg.direct_solve_dual(A64, b.astype(np.float64), p.nu)
    assert linalg.relative_error(A64, p.nu, x, xs) <= 1e-5
    _, ref = oracle_ihs.adaptive_ihs_dual(A64, b.astype(np.float64), p.nu, kind=kind, tol=1e-8)
    assert_same_schedule(ctx.trace(), ref.trace, kind)


def test_dual_spectral(ctx, torch_cuda):
    p = problems.spectral(n=16384, d=512, de_target=40.0, seed=1)
    A = np.ascontiguousarray(p.A.T)                       # 512 x 16384
    b = np.random.default_rng(2).standard_normal(A.shape[0]).astype(np.float32)
    A64 = A.astype(np.float64)
    rep, x = _run(ctx, torch_cuda, A, b, p.nu, "srht", 1e-7)
    assert rep.status == 0
    xs = linalg.direct_solve_dual(A64, b.astype(np.float64), p.nu)
    assert linalg.relative_error(A64, p.nu, x, xs) <= 1e-5
    _, ref = oracle_ihs.adaptive_ihs_dual(A64, b.astype(np.float64), p.nu, kind="srht", tol=1e-7)
    assert_same_schedule(ctx.trace(), ref.trace, "srht")


@pytest.mark.parametrize("n,d", [(250, 3001), (37, 37), (1, 500)])
def test_dual_ragged_and_edge_shapes(ctx, torch_cuda, n, d):
    rng = np.random.default_rng(n + d)
    A = (rng.standard_normal((n, d)) / np.sqrt(d)).astype(np.float32)
    b = rng.standard_normal(n).astype(np.float32)
    nu = 0.3
    rep, x = _run(ctx, torch_cuda, A, b, nu, "srht", 1e-7)
    assert rep.status == 0
    A64 = A.astype(np.float64)
    xs = linalg.direct_solve_dual(A64, b.astype(np.float64), nu)
    assert linalg.relative_error(A64, nu, x, xs) <= 1e-5


def test_dual_rejects_bad_args(ctx, torch_cuda):
    from paper_2006_05874_gb300 import ihs

    torch = torch_cuda
    A = torch.zeros(8, 4, device="cuda")   # n > d: the primal solver's case
    with pytest.raises(ihs.IHSError) as e:
        ctx.solve_dual(A, torch.zeros(8, device="cuda"), 1.0, torch.zeros(4, device="cuda"))
    assert e.value.status == ihs.IHS_EINVAL
    with pytest.raises(ihs.IHSError):
        ctx.solve_dual(torch.zeros(4, 8, device="cuda"), torch.zeros(4, device="cuda"), 0.0,
                       torch.zeros(8, device="cuda"))
