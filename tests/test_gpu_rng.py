"""Bit-exact parity of the SRHT random draws (signs, row subset) with the oracle."""
import numpy as np
import pytest

from oracle import rng

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("n_pad", [1, 1000, 4096, 1 << 17])
@pytest.mark.parametrize("seed,level", [(0, 0), (12345, 3), ((1 << 40) + 7, 11)])
def test_signs_bit_exact(ctx, torch_cuda, n_pad, seed, level):
    torch = torch_cuda
    eps = torch.empty(n_pad, dtype=torch.int8, device="cuda")
    ctx.srht_signs(n_pad, seed, level, eps)
    assert np.array_equal(eps.cpu().numpy(), rng.signs(n_pad, seed, level))


@pytest.mark.parametrize("n_pad,m", [(64, 1), (64, 64), (1000, 37), (4096, 300), (4096, 4095),
                                     (131072, 1024), (1 << 20, 5000), (131072, 1), (131072, 16),
                                     (1 << 20, 6144), (1 << 20, 6145), (9000, 8000), (1 << 22, 3000),
                                     (8193, 2)])
@pytest.mark.parametrize("seed,level", [(0, 0), (99, 7)])
def test_rows_bit_exact(ctx, torch_cuda, n_pad, m, seed, level):
    torch = torch_cuda
    rows = torch.full((m,), -1, dtype=torch.int32, device="cuda")
    ctx.srht_rows(n_pad, m, seed, level, rows)
    assert np.array_equal(rows.cpu().numpy().astype(np.int64), rng.select_rows(n_pad, m, seed, level))


@pytest.mark.parametrize("n_pad,m", [(64, 64), (4096, 300), (131072, 1), (131072, 1000), (20000, 6144)])
def test_rows_exact_fallback(ctx, torch_cuda, monkeypatch, n_pad, m):
    """The single-CTA fallback of the threshold selection (bisection for the
    m-th smallest key, then a direct compaction) gives the same rows."""
    torch = torch_cuda
    monkeypatch.setenv("IHS_SELECT_FORCE_FALLBACK", "1")
    rows = torch.full((m,), -1, dtype=torch.int32, device="cuda")
    ctx.srht_rows(n_pad, m, 5, 2, rows)
    assert np.array_equal(rows.cpu().numpy().astype(np.int64), rng.select_rows(n_pad, m, 5, 2))


def test_rows_rejects_bad_sizes(ctx, torch_cuda):
    from paper_2006_05874_gb300 import ihs

    torch = torch_cuda
    rows = torch.empty(8, dtype=torch.int32, device="cuda")
    for n_pad, m in ((8, 9), (8, 0), (0, 1)):
        with pytest.raises(ihs.IHSError) as e:
            ctx.srht_rows(n_pad, m, 0, 0, rows)
        assert e.value.status == ihs.IHS_EINVAL
