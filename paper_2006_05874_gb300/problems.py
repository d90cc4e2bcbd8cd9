"""Seeded synthetic ridge problems (inputs only).

These generators build the data (A, b, nu) of the workloads the solver is
measured on.  They hold none of the method's arithmetic and are shared by the
CUDA path's tests and benchmark and by the CPU oracle's checks, which always
receive the very same arrays.

Workloads (shapes follow the synthetic experiments of App. A.1, which stand in
for the paper's MNIST / CIFAR10 runs, absent here):

* ``exp_decay``   - A = G diag(0.95^j), G i.i.d. N(0,1), j = 1..d; x0 ~ N(0, I);
                    b = A x0 + noise N(0, I) (4096 x 256, nu = 0.1, noise 0.1).
* ``spectral``    - A = U diag(sigma) V^T with Haar-random orthonormal U (n x d)
                    and V (d x d) obtained from QR factorisations of Gaussian
                    matrices; sigma_j = j^-1 (or any given profile); nu chosen so
                    that sum sigma^2 / (sigma^2 + nu^2) hits a target value;
                    x0 ~ N(0, I); b = A x0 + noise N(0, I) (131072 x 2048,
                    target 100, noise 0.01).

A is stored row-major float32 (the precision the solver takes); b float32.
Large instances are generated with torch on a CUDA device when one is given
(QR of a 131072 x 2048 Gaussian matrix is slow on host cores); their values
then depend on that device's generator, and every consumer reads the same
arrays.
"""
import math
from dataclasses import dataclass, field

import numpy as np


@dataclass
class Problem:
    A: np.ndarray            # float32, n x d, row-major
    b: np.ndarray            # float32, n
    nu: float
    name: str
    sigma: np.ndarray = None  # singular values used to build A (None: not known)
    x0: np.ndarray = None
    meta: dict = field(default_factory=dict)

    @property
    def n(self):
        return self.A.shape[0]

    @property
    def d(self):
        return self.A.shape[1]


def exp_decay(n=4096, d=256, nu=0.1, noise=0.1, decay=0.95, seed=0):
    """A with i.i.d. N(0,1) entries, column j scaled by decay^j (j = 1..d)."""
    rng = np.random.default_rng(seed)
    G = rng.standard_normal((n, d))
    A = G * decay ** np.arange(1, d + 1)[None, :]
    x0 = rng.standard_normal(d)
    b = A @ x0 + noise * rng.standard_normal(n)
    return Problem(A=A.astype(np.float32), b=b.astype(np.float32), nu=float(nu),
                   name="exp_decay_%dx%d" % (n, d), x0=x0,
                   meta=dict(decay=decay, noise=noise, seed=seed))


def nu_for_target(sigma, target, lo=1e-12, hi=1e12):
    """nu > 0 with sum sigma^2/(sigma^2+nu^2) == target, by bisection on log nu
    (problem set-up: picks the regularisation of a synthetic instance)."""
    s2 = np.asarray(sigma, dtype=np.float64) ** 2
    if not 0 < target < len(s2):
        raise ValueError("target must lie in (0, d)")
    a, b = math.log(lo), math.log(hi)
    for _ in range(200):
        mid = 0.5 * (a + b)
        nu2 = math.exp(2 * mid)
        val = float(np.sum(s2 / (s2 + nu2)))
        if val > target:
            a = mid
        else:
            b = mid
    return math.exp(0.5 * (a + b))


def poly_sigma(d, power=1.0):
    return np.arange(1, d + 1, dtype=np.float64) ** (-power)


def _haar_numpy(rng, rows, cols):
    q, r = np.linalg.qr(rng.standard_normal((rows, cols)))
    return q * np.sign(np.diag(r))[None, :]


def spectral(n=131072, d=2048, sigma=None, nu=None, de_target=100.0, noise=0.01, seed=0,
             device=None):
    """A = U diag(sigma) V^T (Haar U, V), nu set for a target
    sum sigma^2/(sigma^2+nu^2) unless given."""
    sigma = poly_sigma(d) if sigma is None else np.asarray(sigma, dtype=np.float64)
    if nu is None:
        nu = nu_for_target(sigma, de_target)
    if device is None:
        rng = np.random.default_rng(seed)
        U = _haar_numpy(rng, n, d)
        V = _haar_numpy(rng, d, d)
        A = (U * sigma[None, :]) @ V.T
        x0 = rng.standard_normal(d)
        b = A @ x0 + noise * rng.standard_normal(n)
        A32, b32 = A.astype(np.float32), b.astype(np.float32)
    else:
        import torch

        gen = torch.Generator(device=device)
        gen.manual_seed(seed)
        Ug = torch.randn(n, d, generator=gen, device=device, dtype=torch.float64)
        U, R = torch.linalg.qr(Ug)
        U = U * torch.sign(torch.diagonal(R))[None, :]
        del Ug, R
        Vg = torch.randn(d, d, generator=gen, device=device, dtype=torch.float64)
        V, R = torch.linalg.qr(Vg)
        V = V * torch.sign(torch.diagonal(R))[None, :]
        sig = torch.as_tensor(sigma, device=device, dtype=torch.float64)
        A = (U * sig[None, :]) @ V.T
        del U
        x0t = torch.randn(d, generator=gen, device=device, dtype=torch.float64)
        bt = A @ x0t + noise * torch.randn(n, generator=gen, device=device, dtype=torch.float64)
        A32 = A.to(torch.float32).cpu().numpy()
        b32 = bt.to(torch.float32).cpu().numpy()
        x0 = x0t.cpu().numpy()
        del A
    return Problem(A=A32, b=b32, nu=float(nu), name="spectral_%dx%d" % (n, d), sigma=sigma,
                   x0=x0, meta=dict(de_target=de_target, noise=noise, seed=seed))


def random_vector(d, seed, scale=1.0):
    """A float32 N(0, scale^2) vector (test iterates)."""
    return (scale * np.random.default_rng(seed).standard_normal(d)).astype(np.float32)


def random_matrix(rows, cols, seed, scale=1.0):
    """A float32 N(0, scale^2) matrix (stand-alone sketches in factor tests)."""
    return (scale * np.random.default_rng(seed).standard_normal((rows, cols))).astype(np.float32)


# Size grid of the warm-start training and held-out sets: n <= 65536,
# n >= 16 d, n d <= 2^27 (512 MB of A).
WARM_SIZES = tuple((n, d) for n in (2048, 4096, 8192, 16384, 32768, 65536)
                   for d in (32, 64, 128, 256, 512, 1024, 2048) if n >= 16 * d and n * d <= (1 << 27))


def sampled_ridge(seed, device, sizes=WARM_SIZES):
    """One random instance of the warm-start family, built on `device`; the two
    generators of the small and the spectral workloads with their parameters
    drawn at random:

    * "decay" (as ``exp_decay``): A = G diag(q^j), G i.i.d. N(0, 1), q ~ U[0.9, 0.999];
    * "poly"  (as ``spectral``):  A = (G / sqrt(n)) diag(j^-p) V^T, p ~ U[0.5, 1.5],
      V Haar; G / sqrt(n) stands in for the Haar U (its columns are orthonormal
      up to O(sqrt(d / n))), which keeps the generation to one GEMM.

    (n, d) is drawn from `sizes`; nu is set for a target effective dimension
    drawn log-uniformly from [2, d/4] (from the nominal singular values
    sqrt(n) q^j resp. j^-p), but nu >= 1e-3 sigma_1; b = A x0 + 0.01 N(0, I)
    with x0 ~ N(0, I).  Returns (A, b, nu, meta) with A, b float32 torch tensors
    on the device."""
    import torch

    rng = np.random.default_rng(seed)
    n, d = sizes[int(rng.integers(len(sizes)))]
    j = np.arange(1, d + 1, dtype=np.float64)
    if rng.random() < 0.5:
        q = float(rng.uniform(0.9, 0.999))
        col = q ** j
        sigma = math.sqrt(n) * col
        fam = "decay%.4f" % q
    else:
        pw = float(rng.uniform(0.5, 1.5))
        sigma = j ** (-pw)
        fam = "poly%.3f" % pw
    hi = max(2.5, d / 4.0)
    target = float(math.exp(rng.uniform(math.log(2.0), math.log(hi))))
    nu = nu_for_target(sigma, target)
    if nu < 1e-3 * sigma[0]:
        # keep (sigma_1 / nu)^2 <= 1e6: a float32 A cannot carry a sharper problem
        nu = 1e-3 * float(sigma[0])
        target = float(np.sum(sigma ** 2 / (sigma ** 2 + nu * nu)))
    gen = torch.Generator(device=device)
    gen.manual_seed(int(rng.integers(1 << 62)))
    G = torch.randn(n, d, generator=gen, device=device, dtype=torch.float32)
    if fam.startswith("decay"):
        A = G * torch.as_tensor(col, device=device, dtype=torch.float32)[None, :]
    else:
        Vg = torch.randn(d, d, generator=gen, device=device, dtype=torch.float64)
        V, R = torch.linalg.qr(Vg)
        V = V * torch.sign(torch.diagonal(R))[None, :]
        M = (torch.as_tensor(sigma, device=device, dtype=torch.float64)[:, None] * V.T).to(torch.float32)
        A = (G @ M) / math.sqrt(n)
    del G
    x0 = torch.randn(d, generator=gen, device=device, dtype=torch.float32)
    b = A @ x0 + 0.01 * torch.randn(n, generator=gen, device=device, dtype=torch.float32)
    return A.contiguous(), b.contiguous(), float(nu), dict(n=n, d=d, family=fam, de_target=target, seed=seed)


def precision_instance(n=1048576, d=4096, scale=300.0, seed=0, device="cuda"):
    """The precision workload's matrix: A = (G / sqrt(n)) diag(sigma) V^T with
    sigma_j = exp(-j / scale), G i.i.d. N(0, 1) (n x d, float32 on the device;
    its columns are orthonormal up to O(sqrt(d / n)), standing in for a Haar U
    that a QR of a 16 GB matrix would give), V Haar (FP64 QR of a d x d Gaussian);
    x0 ~ N(0, I), b = A x0 + 0.01 N(0, I).  Returns (A, b, sigma) with A, b
    float32 torch tensors on the device; nu is chosen by the caller with
    nu_for_target(sigma, d_e)."""
    import torch

    sigma = np.exp(-np.arange(1, d + 1, dtype=np.float64) / scale)
    gen = torch.Generator(device=device)
    gen.manual_seed(seed)
    Vg = torch.randn(d, d, generator=gen, device=device, dtype=torch.float64)
    V, R = torch.linalg.qr(Vg)
    V = V * torch.sign(torch.diagonal(R))[None, :]
    M = (torch.as_tensor(sigma, device=device, dtype=torch.float64)[:, None] * V.T).to(torch.float32)
    del Vg, V, R
    A = torch.empty(n, d, device=device, dtype=torch.float32)
    rows = 65536
    for r0 in range(0, n, rows):
        r1 = min(n, r0 + rows)
        G = torch.randn(r1 - r0, d, generator=gen, device=device, dtype=torch.float32)
        torch.matmul(G, M, out=A[r0:r1])
    A /= math.sqrt(n)
    x0 = torch.randn(d, generator=gen, device=device, dtype=torch.float32)
    b = A @ x0 + 0.01 * torch.randn(n, generator=gen, device=device, dtype=torch.float32)
    return A, b.contiguous(), sigma
