"""The row-sharded path on two gloo ranks (CPU processes): each rank forms its
rows' terms of the gradient and of the sketch with the oracle, `allreduce_sum`
adds them over the ranks, and the sums equal the unsharded oracle values; a
rank-split adaptive IHS (controller replicated on the summed gradient and
sketch) takes the unsharded oracle run's decisions and reaches its solution."""
import os
import socket
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
N, D, NU = 4096, 48, 0.1


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    import torch
    import torch.distributed as dist

    sys.path.insert(0, ROOT)
    from oracle import ihs as oracle_ihs
    from oracle import linalg
    from oracle import sketch as SK
    from paper_2006_05874_gb300 import problems, shard

    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        p = problems.exp_decay(n=N, d=D, seed=3)
        A, b = p.A.astype(np.float64), p.b.astype(np.float64)
        r0, r1 = shard.row_shards(N, world, 1024)[rank]
        mask = np.zeros((N, 1))
        mask[r0:r1] = 1.0

        def summed(v):
            t = torch.from_numpy(np.ascontiguousarray(v, dtype=np.float64))
            return shard.allreduce_sum(t).numpy()

        # this rank's terms, summed over the ranks
        x = np.random.default_rng(1).standard_normal(D)
        Ax = A[r0:r1] @ x
        g_part = np.append(A[r0:r1].T @ (Ax - b[r0:r1]), Ax @ Ax)
        g_sum = summed(g_part)
        sk = {kind: summed(SK.sketch(A * mask, 64, kind, 5, 6)) for kind in ("srht", "gauss")}

        # the rank-split method: exchange the sketch per level, the gradient per pass
        def grad_fn(v):
            Av = A[r0:r1] @ v
            s = summed(np.append(A[r0:r1].T @ (Av - b[r0:r1]), Av @ Av))
            return s[:D] + NU * NU * v, float(s[D])

        def sketch_fn(_A, m, kind, seed, level):
            return summed(SK.sketch(A * mask, m, kind, seed, level))

        res = oracle_ihs.adaptive_ihs(A, b, NU, kind="srht", variant="polyak", tol=1e-8,
                                      grad_fn=grad_fn, sketch_fn=sketch_fn)
        out.put((rank, g_sum, sk, res.trace, res.x))
        dist.barrier()
    finally:
        dist.destroy_process_group()


def test_sharded_terms_and_solve_on_two_gloo_ranks():
    import torch.multiprocessing as mp

    sys.path.insert(0, ROOT)
    from oracle import ihs as oracle_ihs
    from oracle import linalg
    from oracle import sketch as SK
    from paper_2006_05874_gb300 import problems

    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    got = sorted([q.get(timeout=300) for _ in range(2)], key=lambda t: t[0])
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0

    p = problems.exp_decay(n=N, d=D, seed=3)
    A, b = p.A.astype(np.float64), p.b.astype(np.float64)
    x = np.random.default_rng(1).standard_normal(D)
    g_full = linalg.gradient(A, b, 0.0, x)
    ref = oracle_ihs.adaptive_ihs(A, b, NU, kind="srht", variant="polyak", tol=1e-8)
    for rank, g_sum, sk, trace, xs in got:
        assert np.allclose(g_sum[:D], g_full, rtol=1e-12, atol=1e-9 * np.abs(g_full).max())
        assert np.isclose(g_sum[D], float((A @ x) @ (A @ x)), rtol=1e-12)
        for kind in ("srht", "gauss"):
            full = SK.sketch(A, 64, kind, 5, 6)
            assert np.linalg.norm(sk[kind] - full) <= 1e-12 * np.linalg.norm(full)
        # every rank takes the unsharded run's decisions (values equal to rounding)
        assert [e[:3] for e in trace] == [e[:3] for e in ref.trace]
        assert linalg.relative_error(A, NU, xs, ref.x) <= 1e-9
    # and the ranks agree with each other exactly
    assert np.array_equal(got[0][4], got[1][4])
