"""Parity of the factor / apply of H_S^{-1} (Woodbury form for m < d, direct
d x d form for m >= d) and of the sketched Newton decrement with the oracle.

Both sides read the same FP32 SA; the kernels work in FP64 from the exact
FP32 products and round gt to binary32 at the end, so gt matches to a few
binary32 ulps relative to ||gt|| (bound used: 1e-6), and r to 1e-9."""
import numpy as np
import pytest

from oracle import linalg
from paper_2006_05874_gb300 import problems

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("m,d,nu", [(1, 64, 0.1), (7, 64, 0.5), (40, 64, 0.05), (64, 64, 0.1), (200, 64, 0.01),
                                    (33, 100, 1.0), (300, 512, 0.02), (1000, 2048, 0.015), (2048, 256, 0.1)])
def test_apply_parity(ctx, torch_cuda, m, d, nu):
    torch = torch_cuda
    SA = problems.random_matrix(m, d, seed=m * 13 + d, scale=1.0 / np.sqrt(d))
    g = problems.random_vector(d, seed=d)
    F = ctx.factor(torch.from_numpy(SA).cuda(), nu)
    gt = torch.empty(d, device="cuda")
    r = F.apply_hinv(torch.from_numpy(g).cuda(), gt)
    F.destroy()
    ref = linalg.WoodburyFactor(SA, nu)
    gt_ref = ref.apply(g)
    err = np.linalg.norm(gt.cpu().numpy() - gt_ref) / np.linalg.norm(gt_ref)
    assert err <= 1e-6
    r_ref = linalg.newton_decrement(g, gt_ref)
    assert abs(r - r_ref) <= 1e-9 * abs(r_ref)


def test_apply_repeated_and_after_refactor(ctx, torch_cuda):
    torch = torch_cuda
    SA = problems.random_matrix(50, 200, seed=1)
    SAg = torch.from_numpy(SA).cuda()
    F = ctx.factor(SAg, 0.3)
    g = torch.from_numpy(problems.random_vector(200, seed=2)).cuda()
    outs = []
    for _ in range(3):
        gt = torch.empty(200, device="cuda")
        F.apply_hinv(g, gt)
        outs.append(gt.cpu().numpy())
    assert all(np.array_equal(outs[0], o) for o in outs)
    F.destroy()


def test_factor_not_pd(ctx, torch_cuda):
    """A zero row in SA with nu^2 underflowing to 0 gives a zero pivot."""
    from paper_2006_05874_gb300 import ihs

    torch = torch_cuda
    SA = problems.random_matrix(8, 32, seed=3)
    SA[3] = 0.0
    with pytest.raises(ihs.IHSError) as e:
        ctx.factor(torch.from_numpy(SA).cuda(), 1e-170)
    assert e.value.status == ihs.IHS_ENOTPD
    # the context stays usable
    F = ctx.factor(torch.from_numpy(problems.random_matrix(8, 32, seed=4)).cuda(), 0.5)
    F.destroy()


def test_factor_rejects_bad_nu(ctx, torch_cuda):
    from paper_2006_05874_gb300 import ihs

    torch = torch_cuda
    SA = torch.zeros(4, 8, device="cuda")
    for nu in (0.0, -1.0, float("nan")):
        with pytest.raises(ihs.IHSError) as e:
            ctx.factor(SA, nu)
        assert e.value.status == ihs.IHS_EINVAL


def _spectral_sketch(m, d, seed):
    """An m x d sketch-like matrix with the singular values of the spectral
    workload (sigma_j = 1/j, random orthonormal right factor), so that
    K = nu^2 I + SA SA^T (or SA^T SA + nu^2 I) is as ill-conditioned as in the
    solver's own factorisations (kappa ~ 1/nu^2)."""
    g = np.random.default_rng(seed)
    k = min(m, d)
    V, _ = np.linalg.qr(g.standard_normal((d, k)))
    U, _ = np.linalg.qr(g.standard_normal((m, k)))
    s = 1.0 / np.arange(1, k + 1)
    return ((U * s) @ V.T).astype(np.float32)


@pytest.mark.parametrize("m,d,nu", [(1024, 2048, 0.015313), (2048, 2048, 0.015313), (4096, 2048, 0.015313),
                                    (2048, 4096, 0.035637), (8192, 4096, 0.035637)])
def test_apply_parity_solver_sizes(ctx, torch_cuda, m, d, nu):
    """The factor sizes the solver reaches on the spectral workload (k = min(m, d)
    up to 2048, the persistent Cholesky's full size) and on the 1048576 x 4096
    precision workload (k = 4096 at m = 8192), with the workloads' nu."""
    torch = torch_cuda
    SA = _spectral_sketch(m, d, seed=m + d)
    g = problems.random_vector(d, seed=d + 5)
    F = ctx.factor(torch.from_numpy(SA).cuda(), nu)
    gt = torch.empty(d, device="cuda")
    r = F.apply_hinv(torch.from_numpy(g).cuda(), gt)
    F.destroy()
    ref = linalg.WoodburyFactor(SA, nu)
    gt_ref = ref.apply(g)
    err = np.linalg.norm(gt.cpu().numpy() - gt_ref) / np.linalg.norm(gt_ref)
    assert err <= 1e-6, err
    r_ref = linalg.newton_decrement(g, gt_ref)
    assert abs(r - r_ref) <= 1e-9 * abs(r_ref)


@pytest.mark.parametrize("m,d,nu", [(1024, 2048, 0.015313), (2048, 2048, 0.015313), (300, 200, 0.1), (37, 640, 0.2)])
def test_gram_paths_match_oracle(torch_cuda, monkeypatch, m, d, nu):
    """K = X X^T + nu^2 I (App. B.4) on the tensor cores (every entry of SA split
    exactly into three BF16 pieces, slice sums added in double-float) and on the
    CUDA cores (compensated FP32 chains, IHS_GRAM_SIMT=1): each factor's
    application matches the FP64 oracle to the same bounds, and the two agree."""
    from paper_2006_05874_gb300 import ihs

    torch = torch_cuda
    SA = _spectral_sketch(m, d, seed=m + 2 * d)
    g = problems.random_vector(d, seed=d + 9)
    gt_ref = linalg.WoodburyFactor(SA, nu).apply(g)
    r_ref = linalg.newton_decrement(g, gt_ref)
    outs = []
    for simt in ("0", "1"):
        monkeypatch.setenv("IHS_GRAM_SIMT", simt)
        ctx = ihs.Context()
        F = ctx.factor(torch.from_numpy(SA).cuda(), nu)
        gt = torch.empty(d, device="cuda")
        r = F.apply_hinv(torch.from_numpy(g).cuda(), gt)
        F.destroy()
        ctx.destroy()
        gt = gt.cpu().numpy()
        assert np.linalg.norm(gt - gt_ref) / np.linalg.norm(gt_ref) <= 1e-6
        assert abs(r - r_ref) <= 1e-9 * abs(r_ref)
        outs.append(gt)
    assert np.linalg.norm(outs[0] - outs[1]) / np.linalg.norm(gt_ref) <= 2e-6
