"""The allocation-free gradient entry point (ihs_grad_noalloc) against the
regular one (ihs_grad).

ihs_grad_noalloc serves callers that cannot let a library call cudaMalloc or
cudaFree (device memory owned by another allocator, latency-critical loops):
it keeps its scratch in a fixed device array instead of a context.  Both entry
points are called through the C ABI; the new one twice in a row (the second
call runs on the scratch the first one left behind).  It launches the regular
entry point's kernels with the same grid, so on a GPU with at most 160 SMs each
result must equal the regular one bit for bit (elsewhere: agree within the
gradient tests' tolerance), and both must lie within that tolerance of the FP64
oracle's gradient of Eq. 1:
|dg_c| <= 2u|g_c| + 16u ||(r_i a_ic)_i||_2 + 16u nu^2 |x_c|, u = 2^-24.
This file is collected last so that a run stopping at the first failure has
run every other test; it also passes alone in a fresh process.
"""
import numpy as np
import pytest

from oracle import linalg
from paper_2006_05874_gb300 import problems

pytestmark = pytest.mark.gpu
U = 2.0 ** -24


def _tolerance(A, b, nu, x, g_ref):
    A64, b64, x64 = A.astype(np.float64), b.astype(np.float64), x.astype(np.float64)
    r = A64 @ x64 - b64
    scale = np.sqrt((r[:, None] ** 2 * A64 ** 2).sum(axis=0))
    return 2 * U * np.abs(g_ref) + 16 * U * scale + 16 * U * nu * nu * np.abs(x64) + 1e-30


@pytest.mark.parametrize("n,d,nu", [(20000, 512, 0.1), (4099, 256, 0.3), (1000, 2048, 0.015), (300, 8192, 1.0),
                                    (3001, 4096, 0.2), (2049, 1024, 0.05), (777, 3076, 0.5), (5000, 1020, 0.1),
                                    (64, 4, 0.7)])
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
    g_ref32 = g_ref.cpu().numpy()
    g_ref = g_ref32.astype(np.float64)
    g64 = linalg.gradient(A.astype(np.float64), b.astype(np.float64), nu, x.astype(np.float64))
    tol = _tolerance(A, b, nu, x, g64)
    assert np.all(np.abs(g_ref - g64) <= tol), (np.abs(g_ref - g64) / tol).max()
    same_grid = torch.cuda.get_device_properties(0).multi_processor_count <= 160

    for _ in range(2):
        g = torch.full((d,), float("nan"), device="cuda")
        ax2 = torch.full((1,), float("nan"), device="cuda", dtype=torch.float64)
        ihs.grad_noalloc(Ag, bg, nu, xg, g, ax2)
        torch.cuda.synchronize()
        got32 = g.cpu().numpy()
        got = got32.astype(np.float64)
        assert np.all(np.abs(got - g64) <= tol), (np.abs(got - g64) / tol).max()
        if same_grid:
            assert np.array_equal(got32, g_ref32)
            assert float(ax2.item()) == ax2_ref
        else:
            assert np.all(np.abs(got - g_ref) <= 2 * tol)
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
