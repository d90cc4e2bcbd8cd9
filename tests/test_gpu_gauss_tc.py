"""The Gaussian sketch on tcgen05 tensor cores with BF16 operands.

Parity: against the oracle's sketch of the BF16-rounded operands,
(1/sqrt m) bf16(z) bf16(A) in FP64.  Both sides round the same FP32 A; the
kernel's z comes from fast log/sin/cos, a few binary32 ulps from the oracle's,
so a fraction ~2^-12 of the BF16 roundings of z can land on the neighbouring
value (error 2^-8 |z| each): relative Frobenius error ~ 2^-8 sqrt(2^-12) = 6e-5,
plus FP32 accumulation; tolerance 2e-4.  The error against the exact FP64
sketch (BF16 operand rounding, ~2^-9 per product) is stated and bounded by 1e-2.
"""
import numpy as np
import pytest

from oracle import linalg, rng, sketch
from oracle.quant import bf16_round
from paper_2006_05874_gb300 import problems

pytestmark = pytest.mark.gpu
TOL_Q = 2e-4


def _run(torch, A, m, seed, level, precision="bf16"):
    from paper_2006_05874_gb300 import ihs

    ctx = ihs.Context(kind="gauss", precision=precision)
    SA = torch.full((m, A.shape[1]), float("nan"), device="cuda")
    ctx.sketch(torch.from_numpy(np.ascontiguousarray(A)).cuda(), m, "gauss", seed, level, SA)
    out = SA.cpu().numpy().astype(np.float64)
    ctx.destroy()
    return out


def _relfro(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


@pytest.mark.parametrize("n,d,m", [(4096, 256, 1), (4096, 256, 64), (4096, 256, 128), (4096, 256, 300),
                                   (3000, 100, 200), (5000, 300, 129), (64, 512, 16), (20000, 257, 40)])
def test_gauss_bf16_parity(torch_cuda, n, d, m):
    A = problems.random_matrix(n, d, seed=n + d + m)
    got = _run(torch_cuda, A, m, 7, 3)
    ref_q = sketch.gaussian_sketch_bf16(A, m, 7, 3)
    assert _relfro(got, ref_q) <= TOL_Q
    ref = sketch.gaussian_sketch(A, m, 7, 3)
    assert _relfro(got, ref) <= 1e-2     # stated error against the exact FP64 sketch


@pytest.mark.parametrize("n,d,m,precision", [(4096, 1024, 200, "bf16"), (3000, 4096, 64, "bf16"),
                                             (2048, 2048, 130, "bf16"), (4096, 1024, 128, "fp8"),
                                             (1500, 4096, 20, "fp8")])
def test_gauss_wide_parity(torch_cuda, n, d, m, precision):
    """Widths of 2, 4 and 8 column tiles of 512, a partial last tile of sketch
    rows and a ragged last chunk of rows of A, against the oracle's rounded
    sketch."""
    A = problems.random_matrix(n, d, seed=n + 5 * d + m)
    if precision == "fp8":
        A[:, 3] *= 50.0
        got = _run(torch_cuda, A, m, 11, 6, precision="fp8")
        ref_q = sketch.gaussian_sketch_fp8(A, m, 11, 6)
        assert _relfro(got, ref_q) <= 1e-3
    else:
        got = _run(torch_cuda, A, m, 11, 6)
        ref_q = sketch.gaussian_sketch_bf16(A, m, 11, 6)
        assert _relfro(got, ref_q) <= TOL_Q
    # every row of every column tile against the oracle (no tile left unwritten)
    assert np.all(np.isfinite(got))


@pytest.mark.parametrize("n,d,m", [(4096, 256, 1), (4096, 256, 128), (4096, 256, 300), (3000, 100, 200),
                                   (20000, 257, 40)])
def test_gauss_fp8_parity(torch_cuda, n, d, m):
    """E4M3 operands with per-column scales.  Both sides quantise A identically;
    z's E4M3 rounding flips for a fraction ~2^-18 of entries (fast vs libm
    z differ by ~2^-21 relative, E4M3 spacing 2^-3), each flip an error of one
    E4M3 step (2^-3 |z|): relative Frobenius ~ 2^-3 sqrt(2^-18) = 2.4e-4;
    tolerance 1e-3.  Stated error against the exact sketch: E4M3 rounding of
    both operands, bounded by 0.1."""
    A = problems.random_matrix(n, d, seed=n + 2 * d + m)
    A[:, 3] *= 100.0     # columns of very different scales
    A[:, 5] = 0.0        # and a zero column
    got = _run(torch_cuda, A, m, 5, 2, precision="fp8")
    ref_q = sketch.gaussian_sketch_fp8(A, m, 5, 2)
    assert _relfro(got, ref_q) <= 1e-3
    assert np.all(got[:, 5] == 0.0)
    assert _relfro(got, sketch.gaussian_sketch(A, m, 5, 2)) <= 0.1


def test_solve_with_fp8_gaussian_sketch(ctx, torch_cuda):
    torch = torch_cuda
    p = problems.exp_decay(n=4096, d=256, seed=0)
    xs = linalg.direct_solve(p.A, p.b, p.nu)
    ctx.set_params(kind="gauss", variant="gd", precision="fp8", tol=1e-5)
    x = torch.zeros(p.d, device="cuda")
    rep = ctx.solve(torch.from_numpy(p.A).cuda(), torch.from_numpy(p.b).cuda(), p.nu, x)
    assert rep.status == 0
    assert linalg.relative_error(p.A, p.nu, x.cpu().numpy(), xs) <= 1e-5


@pytest.fixture(scope="module")
def full_size_A():
    A = problems.random_matrix(131072, 2048, seed=21, scale=1.0 / 45.0)
    A[:, 7] *= 300.0      # per-column scales matter for FP8
    A[:, 11] *= 1e-3
    return A


@pytest.mark.parametrize("precision,m,tol", [("bf16", 256, TOL_Q), ("bf16", 1024, TOL_Q), ("fp8", 1024, 1e-3)])
def test_gauss_full_size_sampled_rows(torch_cuda, full_size_A, precision, m, tol):
    """131072 x 2048 (the spectral workload's shape, in the launch configuration
    of the solver's settled level m = 1024): sampled rows of SA against the
    oracle's rounded operands, row by row.  FP8: per-column scales from the
    oracle's definition, z and A r rounded to E4M3."""
    from oracle.quant import e4m3_round

    A = full_size_A
    got = _run(torch_cuda, A, m, 2, 8, precision=precision)
    which = [0, 1, m // 2 - 1, m // 2, m - 1]
    z = rng.gaussian_z_rows(which, A.shape[0], 2, 8).astype(np.float32)
    if precision == "bf16":
        ref = (bf16_round(z).astype(np.float64) @ bf16_round(A).astype(np.float64)) / np.sqrt(m)
    else:
        s, r = sketch.fp8_column_scales(A)
        Aq = e4m3_round((A * r[None, :]).astype(np.float32).astype(np.float64))
        ref = (e4m3_round(z.astype(np.float64)) @ Aq) * s.astype(np.float64)[None, :] / np.sqrt(m)
    for k, j in enumerate(which):
        assert _relfro(got[j], ref[k]) <= tol, (j, _relfro(got[j], ref[k]))


def test_solve_with_bf16_gaussian_sketch(ctx, torch_cuda):
    """S only preconditions: the exact FP32-compensated gradient still drives the
    iterate to the FP64 solution."""
    torch = torch_cuda
    p = problems.exp_decay(n=4096, d=256, seed=0)
    xs = linalg.direct_solve(p.A, p.b, p.nu)
    ctx.set_params(kind="gauss", variant="gd", precision="bf16", tol=1e-5)
    x = torch.zeros(p.d, device="cuda")
    rep = ctx.solve(torch.from_numpy(p.A).cuda(), torch.from_numpy(p.b).cuda(), p.nu, x)
    assert rep.status == 0
    assert linalg.relative_error(p.A, p.nu, x.cpu().numpy(), xs) <= 1e-5
