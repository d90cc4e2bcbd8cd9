"""Nested sketches on the GPU (every level keyed like level 0): the row-range
Gaussian sketch against the oracle's rows, the prefix property, and nested
solves against the oracle's nested run."""
import numpy as np
import pytest

from oracle import ihs as oracle_ihs
from oracle import linalg, sketch
from paper_2006_05874_gb300 import problems
from schedule_parity import assert_same_schedule

pytestmark = pytest.mark.gpu


def _relfro(a, b):
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)


@pytest.mark.parametrize("m,row0,mrows", [(64, 32, 32), (100, 4, 96), (256, 128, 128), (1000, 500, 500)])
def test_sketch_rows_fp32_matches_oracle(ctx, torch_cuda, m, row0, mrows):
    torch = torch_cuda
    A = problems.random_matrix(3000, 130, seed=m + row0)
    out = torch.full((mrows, A.shape[1]), float("nan"), device="cuda")
    ctx.set_params(precision="fp32")
    ctx.sketch_rows(torch.from_numpy(A).cuda(), m, 7, 0, row0, mrows, out)
    ref = sketch.gaussian_sketch(A, m, 7, 0)[row0:row0 + mrows]
    assert _relfro(out.cpu().numpy().astype(np.float64), ref) <= 1e-5


def test_sketch_rows_bf16_matches_oracle(ctx, torch_cuda):
    torch = torch_cuda
    A = problems.random_matrix(4096, 256, seed=5)
    m, row0, mrows = 512, 256, 256
    out = torch.empty((mrows, 256), device="cuda")
    ctx.set_params(precision="bf16")
    try:
        ctx.sketch_rows(torch.from_numpy(A).cuda(), m, 3, 0, row0, mrows, out)
    finally:
        ctx.set_params(precision="fp32")
    ref = sketch.gaussian_sketch_bf16(A, m, 3, 0)[row0:row0 + mrows]
    assert _relfro(out.cpu().numpy().astype(np.float64), ref) <= 2e-4


def test_gpu_prefix_property(ctx, torch_cuda):
    torch = torch_cuda
    A = torch.from_numpy(problems.random_matrix(5000, 96, seed=9)).cuda()
    s64 = torch.empty(64, 96, device="cuda")
    s128 = torch.empty(128, 96, device="cuda")
    ctx.sketch(A, 64, "gauss", 4, 0, s64)
    ctx.sketch(A, 128, "gauss", 4, 0, s128)
    a = (s128[:64] * np.sqrt(2.0)).cpu().numpy().astype(np.float64)
    assert _relfro(a, s64.cpu().numpy().astype(np.float64)) <= 1e-6


@pytest.mark.parametrize("kind", ["gauss", "srht"])
def test_nested_solve_matches_oracle(ctx, torch_cuda, kind):
    torch = torch_cuda
    p = problems.exp_decay(n=4096, d=256, seed=0)
    xs = linalg.direct_solve(p.A, p.b, p.nu)
    ctx.set_params(kind=kind, variant="gd", tol=1e-5, nested=1, m_init=1)
    try:
        x = torch.zeros(p.d, device="cuda")
        rep = ctx.solve(torch.from_numpy(p.A).cuda(), torch.from_numpy(p.b).cuda(), p.nu, x)
    finally:
        ctx.set_params(nested=0)
    assert rep.status == 0
    assert linalg.relative_error(p.A, p.nu, x.cpu().numpy(), xs) <= 1e-5
    ref = oracle_ihs.adaptive_ihs(p.A, p.b, p.nu, kind=kind, variant="gd", tol=1e-5, nested=True)
    assert_same_schedule(ctx.trace(), ref.trace, kind)


def test_nested_bf16_solve_accuracy(ctx, torch_cuda):
    torch = torch_cuda
    p = problems.spectral(n=16384, d=512, de_target=40.0, seed=1)
    xs = linalg.direct_solve(p.A, p.b, p.nu)
    ctx.set_params(kind="gauss", variant="gd", precision="bf16", tol=1e-6, nested=1, m_init=1)
    try:
        x = torch.zeros(p.d, device="cuda")
        rep = ctx.solve(torch.from_numpy(p.A).cuda(), torch.from_numpy(p.b).cuda(), p.nu, x)
    finally:
        ctx.set_params(nested=0, precision="fp32", kind="srht")
    assert rep.status == 0
    assert linalg.relative_error(p.A, p.nu, x.cpu().numpy(), xs) <= 1e-5


def test_sketch_rows_rejects_bad_ranges(ctx, torch_cuda):
    from paper_2006_05874_gb300 import ihs

    torch = torch_cuda
    A = torch.zeros(100, 8, device="cuda")
    out = torch.zeros(64, 8, device="cuda")
    for m, row0, mrows in ((64, 2, 8), (64, 60, 8), (64, 0, 0), (64, -4, 8)):
        with pytest.raises(ihs.IHSError) as e:
            ctx.sketch_rows(A, m, 0, 0, row0, mrows, out)
        assert e.value.status == ihs.IHS_EINVAL
