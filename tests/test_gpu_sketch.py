"""Parity of the sketches SA with the FP64 oracle: relative Frobenius error
<= 1e-5 on FP32 SA (the accuracy target of the solver's specification)."""
import numpy as np
import pytest

from oracle import rng, sketch
from oracle.hadamard import next_pow2
from paper_2006_05874_gb300 import problems

pytestmark = pytest.mark.gpu
TOL = 1e-5


def _sketch(torch, ctx, A, m, kind, seed, level):
    Ag = torch.from_numpy(np.ascontiguousarray(A)).cuda()
    SA = torch.full((m, A.shape[1]), float("nan"), dtype=torch.float32, device="cuda")
    ctx.sketch(Ag, m, kind, seed, level, SA)
    return SA.cpu().numpy().astype(np.float64)


def _relfro(a, b):
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)


@pytest.mark.parametrize("n,d,m", [(4096, 256, 1), (4096, 256, 7), (4096, 256, 64), (4096, 256, 300),
                                   (3000, 100, 512), (100, 37, 16), (4096, 256, 2048), (4096, 64, 4096),
                                   (5000, 48, 33), (1, 8, 1), (3000, 100, 200), (4096, 64, 1100),
                                   (2048, 80, 256), (1025, 32, 17)])
@pytest.mark.parametrize("seed,level", [(0, 3), (77, 0)])
def test_srht_parity(ctx, torch_cuda, n, d, m, seed, level):
    A = problems.random_matrix(n, d, seed=n * 7 + d)
    if m > next_pow2(n):
        pytest.skip("m above n_pad")
    got = _sketch(torch_cuda, ctx, A, m, "srht", seed, level)
    ref = sketch.srht_sketch(A, m, seed, level)
    assert _relfro(got, ref) <= TOL


@pytest.mark.parametrize("n,d,m", [(4096, 256, 1), (4096, 256, 5), (4096, 256, 64), (2000, 130, 300),
                                   (100, 37, 16), (1, 8, 3)])
def test_gauss_parity(ctx, torch_cuda, n, d, m):
    A = problems.random_matrix(n, d, seed=n + 3 * d)
    got = _sketch(torch_cuda, ctx, A, m, "gauss", 5, 2)
    ref = sketch.gaussian_sketch(A, m, 5, 2)
    assert _relfro(got, ref) <= TOL


def test_srht_full_size_sampled_rows(ctx, torch_cuda):
    """131072 x 2048 with m = 1024: sampled rows against explicit +-1 sums."""
    A = problems.random_matrix(131072, 2048, seed=11, scale=1.0 / 45.0)
    m = 1024
    got = _sketch(torch_cuda, ctx, A, m, "srht", 0, 10)
    which = [0, 1, 255, 511, 700, 1023]
    ref = sketch.srht_rows_explicit(A, m, 0, 10, which=which)
    for k, j in enumerate(which):
        assert _relfro(got[j], ref[k]) <= TOL


@pytest.mark.parametrize("m,which", [(16, [0, 7, 15]), (200, [0, 99, 199]), (2048, [0, 1023, 1024, 1500, 2047])])
def test_srht_full_size_small_m_sampled_rows(ctx, torch_cuda, m, which):
    """131072 x 2048 at the sketch sizes of the first levels (512-row block
    kernel) and of the last one (m = 2048, one pass with 64 accumulators per
    thread): sampled rows against explicit +-1 sums."""
    A = problems.random_matrix(131072, 2048, seed=14, scale=1.0 / 45.0)
    got = _sketch(torch_cuda, ctx, A, m, "srht", 0, 4)
    ref = sketch.srht_rows_explicit(A, m, 0, 4, which=which)
    for k, j in enumerate(which):
        assert _relfro(got[j], ref[k]) <= TOL


def test_gauss_full_size_sampled_rows(ctx, torch_cuda):
    A = problems.random_matrix(131072, 2048, seed=12, scale=1.0 / 45.0)
    m = 64
    got = _sketch(torch_cuda, ctx, A, m, "gauss", 3, 6)
    which = [0, 5, 63]
    z = rng.gaussian_z_rows(which, 131072, 3, 6)
    ref = (z @ A.astype(np.float64)) / np.sqrt(m)
    for k, j in enumerate(which):
        assert _relfro(got[j], ref[k]) <= TOL


def test_sketch_deterministic(ctx, torch_cuda):
    A = problems.random_matrix(8192, 256, seed=13)
    a = _sketch(torch_cuda, ctx, A, 200, "srht", 1, 8)
    b = _sketch(torch_cuda, ctx, A, 200, "srht", 1, 8)
    assert np.array_equal(a, b)
