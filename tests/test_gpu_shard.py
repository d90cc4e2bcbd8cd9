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


def _full_sketch(ctx, torch, A, m, kind, seed, level):
    SA = torch.full((m, A.shape[1]), float("nan"), device="cuda")
    ctx.sketch(A, m, kind, seed, level, SA)
    return SA.double()


@pytest.mark.parametrize("kind,precision,n,d,m,parts", [
    ("srht", "fp32", 131072, 2048, 16, 4), ("srht", "fp32", 131072, 2048, 1024, 3),
    ("srht", "fp32", 70000, 256, 300, 2), ("srht", "fp32", 5000, 100, 64, 3),
    ("gauss", "fp32", 20000, 300, 128, 3), ("gauss", "bf16", 65536, 1024, 256, 4)])
def test_sketch_by_row_shards(torch_cuda, kind, precision, n, d, m, parts):
    """Each shard's term (global signs, parities and Gaussian columns) summed
    over the shards equals the sketch of the whole matrix, to the FP32
    accumulation order."""
    from paper_2006_05874_gb300 import ihs

    torch = torch_cuda
    ctx = ihs.Context(kind=kind, precision=precision)
    try:
        A = torch.from_numpy(problems.random_matrix(n, d, seed=n + m, scale=1.0 / np.sqrt(d))).cuda()
        full = _full_sketch(ctx, torch, A, m, kind, 9, 4)
        total = torch.zeros(m, d, dtype=torch.float64, device="cuda")
        for r0, r1 in shard.row_shards(n, parts, 1024):
            part = torch.full((m, d), float("nan"), device="cuda")
            ctx.sketch_shard(A[r0:r1], r0, n, m, kind, 9, 4, part)
            total += part.double()
        tol = 2e-4 if precision == "bf16" else 1e-5
        assert torch.linalg.norm(total - full) <= tol * torch.linalg.norm(full)
    finally:
        ctx.destroy()


def test_sketch_shard_rejects_unaligned_srht_rows(ctx, torch_cuda):
    from paper_2006_05874_gb300 import ihs

    torch = torch_cuda
    A = torch.zeros(3000, 64, device="cuda")
    part = torch.zeros(16, 64, device="cuda")
    with pytest.raises(ihs.IHSError):
        ctx.sketch_shard(A[100:2000], 100, 3000, 16, "srht", 0, 0, part)   # row0 off a block
    with pytest.raises(ihs.IHSError):
        ctx.sketch_shard(A[0:1500], 0, 3000, 16, "srht", 0, 0, part)       # ends inside a block


def test_grad_shard_fp64_terms(ctx, torch_cuda):
    torch = torch_cuda
    n, d, nu = 70000, 1024, 0.3
    A = torch.from_numpy(problems.random_matrix(n, d, seed=5, scale=1.0 / np.sqrt(d))).cuda()
    gen = np.random.default_rng(6)
    b = torch.from_numpy(gen.standard_normal(n).astype(np.float32)).cuda()
    x = torch.from_numpy(gen.standard_normal(d).astype(np.float32)).cuda()
    g_full = torch.empty(d, device="cuda")
    ax2_full = ctx.grad(A, b, nu, x, g_full)
    total = torch.zeros(d + 1, dtype=torch.float64, device="cuda")
    for r0, r1 in shard.row_shards(n, 3, 1024):
        gp = torch.full((d + 1,), float("nan"), dtype=torch.float64, device="cuda")
        ctx.grad_shard(A[r0:r1], b[r0:r1], x, gp)
        total += gp
    g = (total[:d] + nu * nu * x.double()).float()
    assert torch.linalg.norm(g.double() - g_full.double()) <= 1e-6 * torch.linalg.norm(g_full.double())
    assert float(total[d]) == pytest.approx(ax2_full, rel=1e-10)


def _emulated_ranks(torch, ihs, A, b, nu, parts, kind, variant, tol):
    """ihs_solve_sharded on `parts` ranks emulated by host threads on one GPU:
    the exchange callback sums the ranks' device buffers on the host in rank
    order (every rank gets the same sums).  All ranks' contexts share one
    stream, so their kernels never run side by side; no kernel of one rank
    waits on another's."""
    import threading

    n, d = A.shape
    shards = shard.row_shards(n, parts, 1024)
    world = len(shards)
    slots = [None] * world
    barrier = threading.Barrier(world)
    stream = torch.cuda.current_stream()
    results = [None] * world
    errors = []

    def make_cb(rank):
        def reduce_fn(t):
            torch.cuda.synchronize()          # every rank's work on the shared stream is done
            slots[rank] = t.cpu().numpy().copy()
            barrier.wait(timeout=60)
            total = slots[0].copy()
            for r in range(1, world):         # rank order: every rank forms the same sums
                total += slots[r]
            t.copy_(torch.from_numpy(total).to(t.device))
            torch.cuda.synchronize()
            barrier.wait(timeout=60)
        return shard.make_allreduce(reduce_fn)

    def run(rank):
        try:
            r0, r1 = shards[rank]
            ctx = ihs.Context(kind=kind, variant=variant, tol=tol, stream=stream)
            x = torch.zeros(d, device="cuda")
            cb = make_cb(rank)
            rep = ctx.solve_sharded(A[r0:r1], b[r0:r1], r0, n, nu, x, cb, tol=tol)
            results[rank] = (rep, ctx.trace(), x.clone())
            torch.cuda.current_stream().synchronize()
            ctx.destroy()
        except Exception as e:   # surfaced below
            errors.append(e)
            barrier.abort()

    threads = [threading.Thread(target=run, args=(r,)) for r in range(world)]
    for t in threads:
        t.start()
    for t in threads:
        t.join(timeout=600)
    assert not errors, errors
    return results


@pytest.mark.parametrize("kind,variant,parts", [("srht", "gd", 2), ("srht", "polyak", 4), ("gauss", "gd", 3)])
def test_solve_on_emulated_row_shards(ctx, torch_cuda, kind, variant, parts):
    """The rank-split solve: every rank takes the decisions of the unsharded
    solve (to the schedule-tie rule), returns the same x as the others, and that
    x meets the FP64 direct solution at 1e-5."""
    from oracle import linalg
    from paper_2006_05874_gb300 import ihs
    from schedule_parity import assert_same_schedule

    torch = torch_cuda
    p = problems.spectral(n=16384, d=512, de_target=40.0, seed=2)
    A, b = torch.from_numpy(p.A).cuda(), torch.from_numpy(p.b).cuda()
    ctx.set_params(kind=kind, variant=variant, tol=1e-5)
    x1 = torch.zeros(p.d, device="cuda")
    rep1 = ctx.solve(A, b, p.nu, x1)
    single = ctx.trace()
    assert rep1.status == 0
    results = _emulated_ranks(torch, ihs, A, b, p.nu, parts, kind, variant, 1e-5)
    xs = linalg.direct_solve(p.A, p.b, p.nu)
    for rep, trace, x in results:
        assert rep.status == 0
        assert_same_schedule(trace, single, kind)
        assert torch.equal(x, results[0][2])
        assert linalg.relative_error(p.A, p.nu, x.cpu().numpy(), xs) <= 1e-5
