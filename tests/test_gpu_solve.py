"""End-to-end adaptive IHS on the GPU against the FP64 oracle: the solution
within 1e-5 relative prediction-norm error of the direct solution, and the
doubling schedule equal to the oracle's run of the same draws."""
import numpy as np
import pytest

from oracle import ihs as oracle_ihs
from oracle import linalg
from paper_2006_05874_gb300 import problems
from schedule_parity import assert_same_schedule

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def exp_problem():
    p = problems.exp_decay(n=4096, d=256, seed=0)
    return p, linalg.direct_solve(p.A, p.b, p.nu)


@pytest.mark.parametrize("kind", ["srht", "gauss"])
@pytest.mark.parametrize("variant", ["gd", "polyak"])
def test_solve_exp_decay(ctx, torch_cuda, exp_problem, kind, variant):
    torch = torch_cuda
    p, xs = exp_problem
    ctx.set_params(kind=kind, variant=variant, tol=1e-5)
    x = torch.zeros(p.d, device="cuda")
    rep = ctx.solve(torch.from_numpy(p.A).cuda(), torch.from_numpy(p.b).cuda(), p.nu, x)
    assert rep.status == 0
    err = linalg.relative_error(p.A, p.nu, x.cpu().numpy(), xs)
    assert err <= 1e-5
    ref = oracle_ihs.adaptive_ihs(p.A, p.b, p.nu, kind=kind, variant=variant, tol=1e-5)
    assert_same_schedule(ctx.trace(), ref.trace, kind)


def test_solve_spectral_small(ctx, torch_cuda):
    torch = torch_cuda
    p = problems.spectral(n=16384, d=512, de_target=40.0, seed=1)
    xs = linalg.direct_solve(p.A, p.b, p.nu)
    ctx.set_params(kind="srht", variant="gd", tol=1e-5)
    x = torch.zeros(p.d, device="cuda")
    rep = ctx.solve(torch.from_numpy(p.A).cuda(), torch.from_numpy(p.b).cuda(), p.nu, x)
    assert rep.status == 0
    assert linalg.relative_error(p.A, p.nu, x.cpu().numpy(), xs) <= 1e-5
    ref = oracle_ihs.adaptive_ihs(p.A, p.b, p.nu, kind="srht", variant="gd", tol=1e-5)
    assert_same_schedule(ctx.trace(), ref.trace, "srht")


def test_solve_warm_start_level(ctx, torch_cuda, exp_problem):
    torch = torch_cuda
    p, xs = exp_problem
    ctx.set_params(kind="srht", variant="gd", tol=1e-5, m_init=512)
    x = torch.zeros(p.d, device="cuda")
    rep = ctx.solve(torch.from_numpy(p.A).cuda(), torch.from_numpy(p.b).cuda(), p.nu, x)
    assert rep.levels()[0] == 512
    assert linalg.relative_error(p.A, p.nu, x.cpu().numpy(), xs) <= 1e-5


def test_solve_rejects_bad_args(ctx, torch_cuda):
    from paper_2006_05874_gb300 import ihs

    torch = torch_cuda
    A = torch.zeros(4, 8, device="cuda")   # n < d
    with pytest.raises(ihs.IHSError):
        ctx.solve(A, torch.zeros(4, device="cuda"), 1.0, torch.zeros(8, device="cuda"))


def test_trace_file_matches_events(ctx, torch_cuda, exp_problem, tmp_path):
    import json

    torch = torch_cuda
    p, _ = exp_problem
    path = tmp_path / "trace.jsonl"
    ctx.set_params(kind="srht", variant="polyak", tol=1e-5, m_init=1)
    ctx.set_trace_file(path)
    try:
        x = torch.zeros(p.d, device="cuda")
        ctx.solve(torch.from_numpy(p.A).cuda(), torch.from_numpy(p.b).cuda(), p.nu, x)
    finally:
        ctx.set_trace_file(None)
    lines = [json.loads(line) for line in path.read_text().splitlines()]
    events = ctx.trace()
    assert len(lines) == len(events) > 0
    for rec, ev in zip(lines, events):
        assert (rec["event"], rec["t"], rec["m"]) == ev[:3]
        assert rec["ratio"] == ev[3]
    assert events[-1][0] == "stop" and events[-1][3] <= 1.0


@pytest.mark.parametrize("variant", ["gd", "polyak"])
def test_resume_reproduces_uninterrupted_run(ctx, torch_cuda, exp_problem, variant):
    """A run stopped by max_iter and resumed from its state takes the same
    decisions and returns the same bits as one uninterrupted run (keyed sketches,
    deterministic kernels)."""
    torch = torch_cuda
    p, xs = exp_problem
    A, b = torch.from_numpy(p.A).cuda(), torch.from_numpy(p.b).cuda()
    ctx.set_params(kind="srht", variant=variant, tol=1e-5, m_init=1, max_iter=500)
    x_full = torch.zeros(p.d, device="cuda")
    rep_full = ctx.solve(A, b, p.nu, x_full)
    full_trace = ctx.trace()
    assert rep_full.status == 0 and rep_full.iterations > 4

    x = torch.zeros(p.d, device="cuda")
    x_prev = torch.zeros(p.d, device="cuda")
    state, pieces = None, []
    for limit in (2, rep_full.iterations // 2 + 1, 500):
        ctx.set_params(kind="srht", variant=variant, tol=1e-5, m_init=1, max_iter=limit)
        rep, state = ctx.solve_resume(A, b, p.nu, x, x_prev, state)
        pieces += ctx.trace()
    assert rep.status == 0
    assert state.t == rep_full.iterations and state.m == rep_full.m_final
    assert state.n_levels >= rep_full.n_levels
    assert pieces == full_trace
    assert torch.equal(x, x_full)
    assert linalg.relative_error(p.A, p.nu, x.cpu().numpy(), xs) <= 1e-5


def test_resume_rejects_inconsistent_state(ctx, torch_cuda):
    from paper_2006_05874_gb300 import ihs

    torch = torch_cuda
    A = torch.zeros(64, 8, device="cuda")
    b = torch.zeros(64, device="cuda")
    x, xp = torch.zeros(8, device="cuda"), torch.zeros(8, device="cuda")
    bad = ihs.State(t=3, level=2, m=8, r1=1.0)          # m != 2^level
    with pytest.raises(ihs.IHSError):
        ctx.solve_resume(A, b, 0.5, x, xp, bad)
    bad = ihs.State(t=3, level=2, m=4, r1=0.0)          # r1 must be positive
    with pytest.raises(ihs.IHSError):
        ctx.solve_resume(A, b, 0.5, x, xp, bad)


@pytest.mark.slow
def test_solve_spectral_full_size_schedule(ctx, torch_cuda):
    """The headline workload itself (131072 x 2048, sigma_j = 1/j, d_e = 100):
    SRHT gradient-IHS from m = 1, decision by decision against the oracle's
    full-size FP64 run of the same draws, and the solution against the FP64
    direct solve (the oracle takes about a minute here)."""
    torch = torch_cuda
    p = problems.spectral(131072, 2048, de_target=100.0, seed=0, device="cuda")
    ctx.set_params(kind="srht", variant="gd", tol=1e-5, m_init=1, max_iter=500)
    x = torch.zeros(p.d, device="cuda")
    rep = ctx.solve(torch.from_numpy(p.A).cuda(), torch.from_numpy(p.b).cuda(), p.nu, x)
    assert rep.status == 0
    events = ctx.trace()
    xs = linalg.direct_solve(p.A, p.b, p.nu)
    assert linalg.relative_error(p.A, p.nu, x.cpu().numpy(), xs) <= 1e-5
    ref = oracle_ihs.adaptive_ihs(p.A, p.b, p.nu, kind="srht", variant="gd", tol=1e-5)
    assert ref.levels[-1] >= 1024
    assert_same_schedule(events, ref.trace, "srht")


def test_solve_host_buffers_match_device_solve(ctx, torch_cuda, exp_problem):
    """ihs_solve_host (host A, b, x; the copies inside the call) returns the
    device-buffer solve's bits, with page-locked and with pageable memory."""
    torch = torch_cuda
    p, xs = exp_problem
    ctx.set_params(kind="srht", variant="gd", tol=1e-5, m_init=1, max_iter=500)
    x_d = torch.zeros(p.d, device="cuda")
    rep_d = ctx.solve(torch.from_numpy(p.A).cuda(), torch.from_numpy(p.b).cuda(), p.nu, x_d)
    for pinned in (True, False):
        A_h, b_h = torch.from_numpy(p.A.copy()), torch.from_numpy(p.b.copy())
        x_h = torch.zeros(p.d)
        if pinned:
            A_h, b_h, x_h = A_h.pin_memory(), b_h.pin_memory(), x_h.pin_memory()
        rep = ctx.solve_host(A_h, b_h, p.nu, x_h)
        assert rep.status == 0 and rep.levels() == rep_d.levels()
        assert torch.equal(x_h, x_d.cpu())
    assert linalg.relative_error(p.A, p.nu, x_h.numpy(), xs) <= 1e-5
