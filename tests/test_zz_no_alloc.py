"""The allocation-free gradient entry point (ihs_grad_noalloc) against the
regular one (ihs_grad).

ihs_grad_noalloc serves callers that cannot let a library call cudaMalloc or
cudaFree (device memory owned by another allocator, latency-critical loops):
it keeps its scratch in a fixed device array instead of a context.  Both entry
points are called through the C ABI; the new one twice in a row (the second
call runs on the scratch the first one left behind), and each result must
agree with the regular entry point within the tolerance of the gradient tests:
|dg_c| <= 2u|g_c| + 16u ||(r_i a_ic)_i||_2 + 16u nu^2 |x_c|, u = 2^-24.
This file is collected last so that a run stopping at the first failure has
run every other test; it also passes alone in a fresh process.
"""
import numpy as np
import pytest

from paper_2006_05874_gb300 import problems

pytestmark = pytest.mark.gpu
U = 2.0 ** -24


def _tolerance(A, b, nu, x, g_ref):
    A64, b64, x64 = A.astype(np.float64), b.astype(np.float64), x.astype(np.float64)
    r = A64 @ x64 - b64
    scale = np.sqrt((r[:, None] ** 2 * A64 ** 2).sum(axis=0))
    return 2 * U * np.abs(g_ref) + 16 * U * scale + 16 * U * nu * nu * np.abs(x64) + 1e-30


@pytest.mark.parametrize("n,d,nu", [(20000, 512, 0.1), (4099, 256, 0.3), (1000, 2048, 0.015), (300, 8192, 1.0)])
def test_noalloc_matches_regular_entry_point(torch_cuda, n, d, nu):
    torch = torch_cuda
    from paper_2006_05874_gb300 import ihs

    A = problems.random_matrix(n, d, seed=n + d)
    b = problems.random_vector(n, seed=n + 1)
    x = problems.random_vector(d, seed=d + 2)
    Ag, bg, xg = (torch.from_numpy(v).cuda() for v in (A, b, x))

    ctx = ihs.Context()
    g_ref = torch.empty(d, device="cuda")
    ax2_ref = ctx.grad(Ag, bg, nu, xg, g_ref)
    ctx.destroy()
    g_ref = g_ref.cpu().numpy().astype(np.float64)
    tol = _tolerance(A, b, nu, x, g_ref)

    for _ in range(2):
        g = torch.full((d,), float("nan"), device="cuda")
        ax2 = torch.full((1,), float("nan"), device="cuda", dtype=torch.float64)
        ihs.grad_noalloc(Ag, bg, nu, xg, g, ax2)
        torch.cuda.synchronize()
        got = g.cpu().numpy().astype(np.float64)
        assert np.all(np.abs(got - g_ref) <= tol), (np.abs(got - g_ref) / tol).max()
        assert abs(float(ax2.item()) - ax2_ref) <= 1e-12 * abs(ax2_ref)


def test_noalloc_rejects_sizes_beyond_limits(torch_cuda):
    torch = torch_cuda
    from paper_2006_05874_gb300 import ihs

    lib = ihs.load()
    for n, d in ((10, 8196), (10, 6), (0, 8)):
        A = torch.zeros(max(n, 1), d, device="cuda")
        v = torch.zeros(max(n, 1), device="cuda")
        x = torch.zeros(d, device="cuda")
        st = lib.ihs_grad_noalloc(None, ihs._ptr(A), ihs._ptr(v), n, d, 0.1, ihs._ptr(x), ihs._ptr(x), None)
        assert st == ihs.IHS_EINVAL
