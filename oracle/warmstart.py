"""Learned warm start of the doubling of m (an addition of this project: the
paper starts Algorithm 1 at m = 1 and allows any initial power of two).

TEST INFRASTRUCTURE ONLY (see the package docstring).

* ``probe_features`` - the 11 features: log n, log d, log nu and
  log sigma_k(P), k in KS, of the Gaussian probe P = S A with S the i.i.d.
  N(0, 1/32) embedding of Sec. 1 at size 32, drawn at level PROBE_LEVEL of
  the seed.  sigma_k(P)^2 are the eigenvalues of P P^T (numpy's symmetric
  eigen-solver stands in for the device's Jacobi sweeps), clamped below at
  1e-10 lambda_1.
* ``forward`` / ``loss_and_grad`` - the 11 -> 64 -> 64 -> 1 tanh network and
  the mean squared error with its gradient by the chain rule, in float64.
* ``adam_step`` - Adam (Kingma & Ba, ICLR 2015, Algorithm 1 of that paper)
  with beta1 0.9, beta2 0.999, eps 1e-8; mu and sd are not updated.
* ``level_from_prediction`` - the initial level 2^clamp(floor(y) - 1, 0,
  floor(log2 n)).

The flat parameter layout (mu, sd, W1, b1, W2, b2, w3, b3) matches the
library's; the oracle keeps its own copy of the offsets.
"""
import math

import numpy as np

from . import sketch as SK

NF, NH = 11, 64
KS = (1, 2, 3, 4, 6, 8, 12, 16)
PROBE_ROWS = 32
PROBE_LEVEL = 200

_SIZES = (("mu", NF), ("sd", NF), ("W1", NH * NF), ("b1", NH), ("W2", NH * NH), ("b2", NH),
          ("w3", NH), ("b3", 1))
OFFSETS = {}
_o = 0
for _name, _sz in _SIZES:
    OFFSETS[_name] = (_o, _sz)
    _o += _sz
NPARAM = _o


def unpack(params):
    """Views of the flat vector as (mu, sd, W1, b1, W2, b2, w3, b3)."""
    p = np.asarray(params, dtype=np.float64)
    out = {}
    for name, (o, sz) in OFFSETS.items():
        out[name] = p[o:o + sz]
    out["W1"] = out["W1"].reshape(NH, NF)
    out["W2"] = out["W2"].reshape(NH, NH)
    out["b3"] = out["b3"][0]
    return out


def pack(mu, sd, W1, b1, W2, b2, w3, b3):
    return np.concatenate([np.ravel(mu), np.ravel(sd), np.ravel(W1), np.ravel(b1), np.ravel(W2),
                           np.ravel(b2), np.ravel(w3), [b3]]).astype(np.float64)


def features_from_gram(Q, n, d, nu):
    """Features from the probe Gram Q = P P^T (32 x 32)."""
    Q = np.asarray(Q, dtype=np.float64)
    lam = np.sort(np.linalg.eigvalsh(0.5 * (Q + Q.T)))[::-1]
    floor = max(lam[0] * 1e-10, 1e-300)
    sig = [0.5 * math.log(max(lam[k - 1], floor)) for k in KS]
    return np.array([math.log(n), math.log(d), math.log(nu)] + sig, dtype=np.float64)


def probe_features(A, nu, seed):
    A = np.asarray(A)
    n, d = A.shape
    P = SK.gaussian_sketch(A, PROBE_ROWS, seed, PROBE_LEVEL)
    return features_from_gram(P @ P.T, n, d, nu)


def forward(params, X, cache=False):
    """y (B,) for features X (B x 11)."""
    w = unpack(params)
    X = np.atleast_2d(np.asarray(X, dtype=np.float64))
    xn = (X - w["mu"][None, :]) / w["sd"][None, :]
    h1 = np.tanh(xn @ w["W1"].T + w["b1"][None, :])
    h2 = np.tanh(h1 @ w["W2"].T + w["b2"][None, :])
    y = h2 @ w["w3"] + w["b3"]
    if cache:
        return y, (xn, h1, h2)
    return y


def loss_and_grad(params, X, target):
    """(1/B) sum (y - t)^2 and its gradient (flat, zero for mu and sd)."""
    w = unpack(params)
    target = np.asarray(target, dtype=np.float64)
    y, (xn, h1, h2) = forward(params, X, cache=True)
    B = y.shape[0]
    e = y - target
    loss = float(e @ e) / B
    dy = 2.0 * e / B                               # dL/dy
    g_w3 = h2.T @ dy
    g_b3 = dy.sum()
    dz2 = (dy[:, None] * w["w3"][None, :]) * (1.0 - h2 * h2)
    g_W2 = dz2.T @ h1
    g_b2 = dz2.sum(axis=0)
    dz1 = (dz2 @ w["W2"]) * (1.0 - h1 * h1)
    g_W1 = dz1.T @ xn
    g_b1 = dz1.sum(axis=0)
    grad = pack(np.zeros(NF), np.zeros(NF), g_W1, g_b1, g_W2, g_b2, g_w3, g_b3)
    return loss, grad


def adam_step(params, m, v, step, grad, lr, beta1=0.9, beta2=0.999, eps=1e-8):
    """Returns (params', m', v'); step is 1-based; mu and sd stay fixed."""
    params = np.array(params, dtype=np.float64)
    m = beta1 * np.asarray(m, dtype=np.float64) + (1.0 - beta1) * grad
    v = beta2 * np.asarray(v, dtype=np.float64) + (1.0 - beta2) * grad * grad
    mhat = m / (1.0 - beta1 ** step)
    vhat = v / (1.0 - beta2 ** step)
    upd = lr * mhat / (np.sqrt(vhat) + eps)
    o = OFFSETS["W1"][0]
    params[o:] -= upd[o:]
    m[:o] = 0.0
    v[:o] = 0.0
    return params, m, v


def level_from_prediction(y, n):
    lvl = int(math.floor(y)) - 1
    cap = int(math.floor(math.log2(n)))
    return 1 << min(max(lvl, 0), cap)
