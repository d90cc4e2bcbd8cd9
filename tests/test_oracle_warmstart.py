"""Pins of the warm-start oracle (probe features, network, Adam) against closed
forms, invariances and finite differences."""
import math

import numpy as np
import pytest

from oracle import warmstart as W


def _orth(k, seed):
    q, r = np.linalg.qr(np.random.default_rng(seed).standard_normal((k, k)))
    return q * np.sign(np.diag(r))[None, :]


def test_layout_size():
    assert W.NPARAM == 11 + 11 + 64 * 11 + 64 + 64 * 64 + 64 + 64 + 1


def test_features_from_gram_known_spectrum():
    lam = 3.0 * 0.7 ** np.arange(32)           # distinct, descending
    U = _orth(32, 1)
    Q = (U * lam[None, :]) @ U.T
    f = W.features_from_gram(Q, n=5000, d=300, nu=0.25)
    assert f[:3] == pytest.approx([math.log(5000), math.log(300), math.log(0.25)], abs=1e-14)
    want = [0.5 * math.log(lam[k - 1]) for k in W.KS]
    assert np.allclose(f[3:], want, atol=1e-9)


def test_features_floor_for_rank_deficient_probe():
    lam = np.zeros(32)
    lam[:3] = [4.0, 2.0, 1.0]
    U = _orth(32, 2)
    f = W.features_from_gram((U * lam[None, :]) @ U.T, 100, 3, 1.0)
    assert f[3:6] == pytest.approx([0.5 * math.log(4.0), 0.5 * math.log(2.0), 0.0], abs=1e-9)
    floor = 0.5 * math.log(4.0 * 1e-10)
    assert np.allclose(f[6:], floor, atol=1e-6)


def test_probe_features_invariances():
    rng = np.random.default_rng(3)
    n, d = 700, 40
    A = rng.standard_normal((n, d)) * (0.8 ** np.arange(d))[None, :]
    f = W.probe_features(A, 0.5, seed=11)
    # right-multiplying A by an orthogonal V leaves P P^T unchanged
    f_rot = W.probe_features(A @ _orth(d, 4), 0.5, seed=11)
    assert np.allclose(f, f_rot, atol=1e-9)
    # scaling A by c shifts every log sigma by log c
    f_sc = W.probe_features(3.0 * A, 0.5, seed=11)
    assert np.allclose(f_sc[3:] - f[3:], math.log(3.0), atol=1e-9)
    # a different level or seed gives a different probe
    assert not np.allclose(f, W.probe_features(A, 0.5, seed=12))


def test_probe_rank_one():
    rng = np.random.default_rng(5)
    u, v = rng.standard_normal(300), rng.standard_normal(20)
    f = W.probe_features(np.outer(u, v), 1.0, seed=0)
    assert np.allclose(f[4:], f[3] + 0.5 * math.log(1e-10), atol=1e-6)


def _random_params(seed, scale=0.3):
    rng = np.random.default_rng(seed)
    p = scale * rng.standard_normal(W.NPARAM)
    o, _ = W.OFFSETS["mu"]
    p[o:o + W.NF] = rng.standard_normal(W.NF)
    o, _ = W.OFFSETS["sd"]
    p[o:o + W.NF] = 0.5 + rng.random(W.NF)
    return p


def test_forward_zero_hidden_weights():
    p = _random_params(6)
    for name in ("W1", "W2"):
        o, sz = W.OFFSETS[name]
        p[o:o + sz] = 0.0
    w = W.unpack(p)
    X = np.random.default_rng(7).standard_normal((3, W.NF))
    want = w["b3"] + sum(w["w3"][k] * math.tanh(w["b2"][k]) for k in range(W.NH))
    assert np.allclose(W.forward(p, X), want, atol=1e-13)


def test_forward_single_path():
    # W1 picks feature 4 into unit 7, W2 = I, w3 = e_7: y = tanh(tanh((x4 - mu4) / sd4))
    mu = np.linspace(-1, 1, W.NF)
    sd = np.linspace(0.5, 2, W.NF)
    W1 = np.zeros((W.NH, W.NF))
    W1[7, 4] = 1.0
    w3 = np.zeros(W.NH)
    w3[7] = 1.0
    p = W.pack(mu, sd, W1, np.zeros(W.NH), np.eye(W.NH), np.zeros(W.NH), w3, 0.0)
    X = np.random.default_rng(8).standard_normal((4, W.NF))
    want = [math.tanh(math.tanh((x[4] - mu[4]) / sd[4])) for x in X]
    assert np.allclose(W.forward(p, X), want, atol=1e-14)


def test_gradient_matches_central_differences():
    p = _random_params(9)
    rng = np.random.default_rng(10)
    X = rng.standard_normal((6, W.NF))
    t = rng.standard_normal(6)
    _, g = W.loss_and_grad(p, X, t)
    h = 1e-6
    idx = list(range(W.OFFSETS["W1"][0], W.NPARAM, 37)) + [W.NPARAM - 1, W.OFFSETS["b1"][0]]
    for i in idx:
        pp, pm = p.copy(), p.copy()
        pp[i] += h
        pm[i] -= h
        fd = (W.loss_and_grad(pp, X, t)[0] - W.loss_and_grad(pm, X, t)[0]) / (2 * h)
        assert abs(fd - g[i]) <= 1e-7 + 1e-6 * abs(fd), i
    assert np.all(g[:2 * W.NF] == 0.0)


def test_adam_constant_gradient_steps():
    # with a constant gradient, the bias-corrected moments are exactly g and g^2,
    # so every step moves by lr g / (|g| + eps)
    p = _random_params(11)
    g = np.random.default_rng(12).standard_normal(W.NPARAM) * 1e-3
    g[:2 * W.NF] = 0.0
    m = np.zeros(W.NPARAM)
    v = np.zeros(W.NPARAM)
    q = p.copy()
    for step in range(1, 6):
        q, m, v = W.adam_step(q, m, v, step, g, lr=1e-2)
    want = p - 5 * 1e-2 * g / (np.abs(g) + 1e-8)
    assert np.allclose(q, want, atol=1e-12, rtol=1e-9)
    assert np.all(q[:2 * W.NF] == p[:2 * W.NF])


def test_adam_reduces_loss_on_a_small_fit():
    rng = np.random.default_rng(13)
    X = rng.standard_normal((64, W.NF))
    t = np.sin(X[:, 0]) + 0.5 * X[:, 3]
    p = _random_params(14, scale=0.1)
    o, _ = W.OFFSETS["mu"]
    p[o:o + W.NF] = 0.0
    o, _ = W.OFFSETS["sd"]
    p[o:o + W.NF] = 1.0
    m = np.zeros(W.NPARAM)
    v = np.zeros(W.NPARAM)
    l0 = W.loss_and_grad(p, X, t)[0]
    for step in range(1, 201):
        _, g = W.loss_and_grad(p, X, t)
        p, m, v = W.adam_step(p, m, v, step, g, lr=3e-3)
    assert W.loss_and_grad(p, X, t)[0] < 0.1 * l0


def test_level_from_prediction():
    assert W.level_from_prediction(10.3, 1 << 20) == 1 << 9
    assert W.level_from_prediction(11.0, 1 << 20) == 1 << 10
    assert W.level_from_prediction(0.5, 100) == 1
    assert W.level_from_prediction(-3.0, 100) == 1
    assert W.level_from_prediction(40.0, 1000) == 512
