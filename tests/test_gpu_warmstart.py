"""Learned warm start on the GPU: probe features, network forward / gradient /
Adam step against the FP64 oracle, the m0 rule, and the gain of the trained
network over the cold doubling from m = 1 on held-out problems."""
import os
import time

import numpy as np
import pytest

from oracle import linalg, warmstart as W
from paper_2006_05874_gb300 import problems

pytestmark = pytest.mark.gpu

WEIGHTS = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "paper_2006_05874_gb300",
                       "warmstart_weights.json")


def _dev(torch, a):
    return torch.as_tensor(np.ascontiguousarray(a, dtype=np.float32), device="cuda")


def _params(seed, scale=0.3):
    rng = np.random.default_rng(seed)
    p = scale * rng.standard_normal(W.NPARAM)
    o, _ = W.OFFSETS["mu"]
    p[o:o + W.NF] = rng.standard_normal(W.NF)
    o, _ = W.OFFSETS["sd"]
    p[o:o + W.NF] = 0.5 + rng.random(W.NF)
    return p.astype(np.float32)


@pytest.mark.parametrize("case", ["exp_decay", "spectral", "rank_deficient", "wide"])
def test_probe_features_parity(ctx, torch_cuda, case):
    torch = torch_cuda
    if case == "exp_decay":
        p = problems.exp_decay(4096, 256, seed=1)
        A, nu = p.A, p.nu
    elif case == "spectral":
        p = problems.spectral(3000, 64, de_target=10.0, seed=2)
        A, nu = p.A, p.nu
    elif case == "rank_deficient":
        A, nu = problems.random_matrix(1500, 8, seed=3), 0.3      # d < 16: floored features
    else:
        A, nu = problems.random_matrix(600, 1000, seed=4, scale=0.1), 2.0
    want = W.probe_features(A, nu, seed=5)
    f = torch.zeros(11, device="cuda", dtype=torch.float32)
    ctx.probe_features(_dev(torch, A), nu, 5, f)
    got = f.cpu().numpy().astype(np.float64)
    assert np.allclose(got[:3], want[:3], atol=1e-6)
    assert np.allclose(got[3:], want[3:], atol=2e-3), (got, want)


@pytest.mark.parametrize("B", [1, 4, 37, 256])
def test_mlp_forward_parity(ctx, torch_cuda, B):
    torch = torch_cuda
    p = _params(10 + B)
    X = np.random.default_rng(B).standard_normal((B, W.NF)).astype(np.float32)
    y = torch.zeros(B, device="cuda", dtype=torch.float32)
    ctx.mlp_forward(_dev(torch, p), _dev(torch, X), y)
    want = W.forward(p.astype(np.float64), X.astype(np.float64))
    assert np.allclose(y.cpu().numpy(), want, atol=2e-5 * max(1.0, np.abs(want).max()))


@pytest.mark.parametrize("B", [3, 37, 256])
def test_mlp_grad_parity(ctx, torch_cuda, B):
    torch = torch_cuda
    p = _params(20 + B)
    rng = np.random.default_rng(30 + B)
    X = rng.standard_normal((B, W.NF)).astype(np.float32)
    t = (5 + 3 * rng.standard_normal(B)).astype(np.float32)
    g = torch.zeros(W.NPARAM, device="cuda", dtype=torch.float32)
    loss = ctx.mlp_grad(_dev(torch, p), _dev(torch, X), _dev(torch, t), g)
    want_loss, want_g = W.loss_and_grad(p.astype(np.float64), X.astype(np.float64), t.astype(np.float64))
    assert loss == pytest.approx(want_loss, rel=1e-5)
    got = g.cpu().numpy().astype(np.float64)
    scale = np.abs(want_g).max()
    assert np.abs(got - want_g).max() <= 1e-5 * scale
    assert np.all(got[:2 * W.NF] == 0.0)


def test_mlp_train_steps_parity(ctx, torch_cuda):
    torch = torch_cuda
    p = _params(40, scale=0.2)
    rng = np.random.default_rng(41)
    X = rng.standard_normal((64, W.NF)).astype(np.float32)
    t = (3 + rng.standard_normal(64)).astype(np.float32)
    pd, md, vd = _dev(torch, p), torch.zeros(W.NPARAM, device="cuda"), torch.zeros(W.NPARAM, device="cuda")
    Xd, td = _dev(torch, X), _dev(torch, t)
    q = p.astype(np.float64)
    m = np.zeros(W.NPARAM)
    v = np.zeros(W.NPARAM)
    lr = 1e-3
    for step in range(1, 4):
        _, g = W.loss_and_grad(q, X.astype(np.float64), t.astype(np.float64))
        loss = ctx.mlp_train_step(pd, md, vd, step, Xd, td, lr)
        assert loss == pytest.approx(W.loss_and_grad(q, X, t)[0], rel=1e-4)
        q, m, v = W.adam_step(q, m, v, step, g, lr)
    got = pd.cpu().numpy().astype(np.float64)
    # steps are ~lr per coordinate; coordinates whose gradient is far above
    # float32 rounding agree to a small fraction of one step
    _, g0 = W.loss_and_grad(p.astype(np.float64), X.astype(np.float64), t.astype(np.float64))
    big = np.abs(g0) > 1e-3 * np.abs(g0).max()
    assert big.sum() > W.NPARAM // 2
    assert np.abs(got - q)[big].max() <= 0.02 * lr
    assert np.abs(got - q).max() <= 3 * 2 * lr
    assert np.all(got[:2 * W.NF] == p[:2 * W.NF])


def test_mlp_rejects_bad_args(ctx, torch_cuda):
    from paper_2006_05874_gb300 import ihs

    torch = torch_cuda
    p = torch.zeros(W.NPARAM, device="cuda")
    X = torch.zeros(0, W.NF, device="cuda")
    with pytest.raises(ihs.IHSError):
        ctx.mlp_forward(p, X, torch.zeros(1, device="cuda"))


@pytest.fixture(scope="module")
def trained():
    from paper_2006_05874_gb300 import warmstart

    if not os.path.exists(WEIGHTS):
        pytest.fail("trained warm-start parameters are missing")
    return warmstart.load_params(WEIGHTS)


def test_weights_file_matches_network(trained, lib):
    params, meta = trained
    assert params.size == lib.ihs_mlp_num_params() == W.NPARAM
    assert np.all(np.isfinite(params))
    assert meta["summary"]["heldout_mse"] < meta["summary"]["heldout_mse_constant"]


@pytest.mark.parametrize("case", [0, 1, 2])
def test_warm_start_m0_matches_oracle(ctx, torch_cuda, trained, case):
    torch = torch_cuda
    params, _ = trained
    p = [problems.exp_decay(4096, 256, seed=3), problems.spectral(8192, 128, de_target=20.0, seed=4),
         problems.exp_decay(16384, 512, decay=0.99, nu=0.01, seed=5)][case]
    m0, pred = ctx.warm_start(_dev(torch, params), _dev(torch, p.A), p.nu, seed=ctx.params.seed)
    f = W.probe_features(p.A, p.nu, ctx.params.seed)
    want_pred = float(W.forward(params.astype(np.float64), f[None, :])[0])
    assert pred == pytest.approx(want_pred, abs=5e-3)
    if abs(want_pred - round(want_pred)) > 5e-3:
        assert m0 == W.level_from_prediction(want_pred, p.n)
    assert m0 & (m0 - 1) == 0 and 1 <= m0 <= p.n


def test_warm_start_gain_on_heldout(ctx, torch_cuda, trained):
    """Held-out problems of the training family (seeds never trained on): the
    warm-started solve reaches the same accuracy with fewer gradient passes and
    less total time (probe and prediction included) than the doubling from m = 1."""
    torch = torch_cuda
    params, _ = trained
    pd = _dev(torch, params)
    sizes = tuple(s for s in problems.WARM_SIZES if s[0] <= 32768)
    cold_t = warm_t = 0.0
    cold_p = warm_p = 0
    for seed in range(950000, 950006):
        A, b, nu, meta = problems.sampled_ridge(seed, "cuda", sizes=sizes)
        d = A.shape[1]
        ctx.set_params(m_init=1)
        x = torch.zeros(d, device="cuda")
        ctx.solve(A, b, nu, x)                       # untimed: caches and arena
        runs = {}
        for mode in ("cold", "warm"):
            best = None
            for _ in range(3):
                x = torch.zeros(d, device="cuda")
                torch.cuda.synchronize()
                t0 = time.perf_counter()
                if mode == "warm":
                    m0, _ = ctx.warm_start(pd, A, nu)
                    ctx.set_params(m_init=m0)
                else:
                    ctx.set_params(m_init=1)
                rep = ctx.solve(A, b, nu, x)
                torch.cuda.synchronize()
                dt = time.perf_counter() - t0
                best = (dt, rep, x) if best is None or dt < best[0] else best
            runs[mode] = best
        ctx.set_params(m_init=1)
        An = A.cpu().numpy()
        xs = linalg.direct_solve(An, b.cpu().numpy(), nu)
        for mode in ("cold", "warm"):
            assert linalg.relative_error(An, nu, runs[mode][2].cpu().numpy(), xs) <= 1e-5, (mode, meta)
        cold_t += runs["cold"][0]
        warm_t += runs["warm"][0]
        cold_p += runs["cold"][1].grad_passes
        warm_p += runs["warm"][1].grad_passes
    assert warm_p < cold_p
    assert warm_t < cold_t, (warm_t, cold_t)


def test_warm_start_batched_matches_single(ctx, torch_cuda, trained):
    torch = torch_cuda
    params, _ = trained
    pd = _dev(torch, params)
    probs = [problems.exp_decay(4096, 256, seed=3), problems.spectral(8192, 128, de_target=20.0, seed=4),
             problems.exp_decay(2048, 64, decay=0.9, nu=1.0, seed=6)]
    dev = [(_dev(torch, p.A), p.nu) for p in probs]
    m0s, preds = ctx.warm_start_batched(pd, dev)
    for (A, nu), m0b, pb in zip(dev, m0s, preds):
        m0, pred = ctx.warm_start(pd, A, nu)
        assert pb == pytest.approx(pred, abs=1e-5)
        assert m0b == m0
