"""The gradient by emulated row shards on one GPU (per-shard passes summed as the
collective would sum them) equals the one-pass gradient."""
import numpy as np
import pytest

from paper_2006_05874_gb300 import problems, shard

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("n,d,parts", [(131072, 2048, 4), (5000, 300, 3), (70000, 1024, 2)])
def test_grad_by_emulated_row_shards(ctx, torch_cuda, n, d, parts):
    torch = torch_cuda
    A = torch.from_numpy(problems.random_matrix(n, d, seed=n + d, scale=1.0 / np.sqrt(d))).cuda()
    gen = np.random.default_rng(d)
    b = torch.from_numpy(gen.standard_normal(n).astype(np.float32)).cuda()
    x = torch.from_numpy(gen.standard_normal(d).astype(np.float32)).cuda()
    nu = 0.3
    g_full = torch.empty(d, device="cuda")
    ax2_full = ctx.grad(A, b, nu, x, g_full)
    sh = shard.row_shards(n, parts, 1024)
    pieces, ax2 = [], 0.0
    for k, (r0, r1) in enumerate(sh):
        g = torch.empty(d, device="cuda")
        ax2 += ctx.grad(A[r0:r1], b[r0:r1], nu if k == 0 else 0.0, x, g)
        pieces.append(g.double())
    g_sh = shard.allreduce_sum(sum(pieces))
    gf = g_full.double()
    assert torch.linalg.norm(g_sh - gf) <= 1e-6 * torch.linalg.norm(gf)
    assert ax2 == pytest.approx(ax2_full, rel=1e-10)
