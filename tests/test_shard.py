"""Row shards and the identity collective (CPU)."""
import numpy as np
import pytest

from paper_2006_05874_gb300 import shard


@pytest.mark.parametrize("n,parts,align", [(1, 1, 1), (10, 3, 1), (131072, 4, 1024), (5000, 3, 1024), (3000, 8, 1024)])
def test_row_shards_partition(n, parts, align):
    sh = shard.row_shards(n, parts, align)
    assert sh[0][0] == 0 and sh[-1][1] == n
    for (a0, a1), (b0, b1) in zip(sh, sh[1:]):
        assert a1 == b0
    assert all(r0 % align == 0 for r0, _ in sh)
    assert len(sh) <= parts


def test_allreduce_is_identity_on_one_rank():
    torch = pytest.importorskip("torch")
    x = torch.arange(5.0)
    assert shard.allreduce_sum(x) is x
    assert torch.equal(x, torch.arange(5.0))


def test_sharded_gradient_algebra_fp64():
    # sum_p A_p^T (A_p x - b_p) + nu^2 x equals the full gradient (the identity the
    # row sharding relies on), with nu^2 x added on shard 0 only
    from oracle import linalg

    rng = np.random.default_rng(0)
    A, b, x = rng.standard_normal((3000, 40)), rng.standard_normal(3000), rng.standard_normal(40)
    nu = 0.7
    parts = [linalg.gradient(A[r0:r1], b[r0:r1], nu if k == 0 else 0.0, x)
             for k, (r0, r1) in enumerate(shard.row_shards(3000, 3, 1024))]
    assert np.allclose(sum(parts), linalg.gradient(A, b, nu, x), rtol=1e-12, atol=1e-10)
