"""Comparators of Sec. 5: conjugate gradient on the normal equations
(A^T A + nu^2 I) x = A^T b, and randomized preconditioned CG (Rokhlin-Tygert
style), whose preconditioner is the sketched Hessian H_S = (SA)^T SA + nu^2 I
of a sketch of size m = ceil(d / rho) (Gaussian) or ceil(d ln d / rho) (SRHT),
capped at n_pad (SRHT) or n (Gaussian).  The paper gives the sketch sizes
(Sec. 5); the preconditioner form and the stopping rule are this project's
reading: stop when ||r|| <= tol ||A^T b||, r = A^T b - (A^T A + nu^2 I) x.
"""
import math

import numpy as np

from . import linalg, sketch as SK
from .hadamard import next_pow2


def pcg_sketch_size(kind, n, d, rho=0.1):
    if kind == "gauss":
        m = math.ceil(d / rho)
        return min(m, n)
    m = math.ceil(d * math.log(d) / rho)
    return min(m, next_pow2(n))


def cg(A, b, nu, tol=1e-8, max_iter=1000, x0=None, precond=None):
    """Preconditioned CG on H x = A^T b with H = A^T A + nu^2 I; precond(v)
    returns M^{-1} v (None: identity).  Returns (x, iterations, residual history)."""
    A = np.asarray(A, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    d = A.shape[1]
    H = lambda v: A.T @ (A @ v) + nu * nu * v
    x = np.zeros(d) if x0 is None else np.asarray(x0, dtype=np.float64).copy()
    atb = A.T @ b
    r = atb - H(x)
    z = precond(r) if precond else r
    p = z.copy()
    rz = r @ z
    norm0 = np.linalg.norm(atb)
    hist = [np.linalg.norm(r)]
    it = 0
    while it < max_iter and hist[-1] > tol * norm0:
        q = H(p)
        alpha = rz / (p @ q)
        x += alpha * p
        r -= alpha * q
        hist.append(np.linalg.norm(r))
        it += 1
        if hist[-1] <= tol * norm0:
            break
        z = precond(r) if precond else r
        rz_new = r @ z
        p = z + (rz_new / rz) * p
        rz = rz_new
    return x, it, hist


def pcg(A, b, nu, kind="srht", rho=0.1, seed=0, tol=1e-8, max_iter=1000):
    """Sketch-preconditioned CG; the sketch is drawn at level 0 of `seed`."""
    n, d = np.asarray(A).shape
    m = pcg_sketch_size(kind, n, d, rho)
    F = linalg.WoodburyFactor(SK.sketch(A, m, kind, seed, 0), nu)
    x, it, hist = cg(A, b, nu, tol=tol, max_iter=max_iter, precond=F.apply)
    return x, it, hist, m
