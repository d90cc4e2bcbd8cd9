"""Adaptive Polyak-IHS (Algorithm 1) and its gradient-only variant (Sec. 5), in
float64, following Algorithm 1's steps in order.

Readings of points the paper leaves open:

* parameters: rho = 0.1, eta = 0.01 by default; cbar_gd = c_gd, cbar_p = c_p
  and the step sizes of Def 3.1 (Gaussian) / Def 3.2 (SRHT), as Thm 4.1 / 4.2
  prescribe;
* the sketch drawn at sketch size m = 2^level is keyed by (seed, level), so a run
  started at m_init = 2^l reproduces the draws of a run started at 1 from level
  l on;
* when Algorithm 1 doubles m and redraws S, it then retries the same t
  starting with the Polyak candidate; both gt_t and r_t are recomputed under
  the new H_S, while r_1 in the Polyak ratio keeps its value from t = 1;
* m is capped at n_pad (SRHT: S is then an orthogonal transform and H_S = H)
  or n (Gaussian); at the cap a rejected gradient step is accepted anyway and
  the run is flagged;
* stopping: before each iteration, stop once sqrt(2 Lambda r_t) <=
  tol * sqrt(||A x_t||^2 + nu^2 ||x_t||^2), because delta_t <= gamma_1 r_t
  <= Lambda r_t (proofs of Thm 4.1 / 4.2) and ||Abar x_t|| estimates ||Abar x*||;
* optional floor guard: a rejected gradient step with r_t <= floor^2 r_1 ends
  the run instead of doubling m (the improvement ratio carries no information
  once the gradient is at the arithmetic's noise floor); floor = 0 disables it.
"""
import math
from dataclasses import dataclass, field

import numpy as np

from . import linalg, params as P, sketch as SK
from .hadamard import next_pow2


@dataclass
class IHSResult:
    x: np.ndarray
    m: int
    level: int
    iterations: int
    status: str
    trace: list = field(default_factory=list)
    levels: list = field(default_factory=list)
    grad_passes: int = 0
    r: float = 0.0
    r1: float = 0.0
    history: list = field(default_factory=list)


def adaptive_ihs(A, b, nu, kind="srht", variant="gd", seed=0, rho=0.1, eta=0.01,
                 m_init=1, x0=None, x1=None, tol=1e-5, max_iter=200, floor=0.0,
                 sketch_fn=None, keep_history=False, dual_b=None, nested=False, grad_fn=None):
    """Run Algorithm 1 (variant="polyak") or its gradient-only variant
    (variant="gd", Sec. 5) on min 1/2||Ax-b||^2 + nu^2/2 ||x||^2.

    sketch_fn(A, m, kind, seed, level) -> SA may replace the oracle's own sketch
    (used to run the method on externally given sketches in tests).
    grad_fn(v) -> (A^T (A v - b) + nu^2 v, ||A v||^2) may replace the oracle's own
    gradient (a rank of a row-sharded run sums its rows' terms with the others').
    keep_history stores (t, x_t, SA in force) for every iterate (small n only).
    dual_b: run on the dual of App. A.2 instead, with A standing for the dual's
    data matrix (the transpose of the primal one) and the gradient
    A^T A z - dual_b + nu^2 z in place of A^T (A z - b) + nu^2 z (b unused).
    nested: every level draws its sketch with the key of level 0, so that the
    sketches are nested: the Gaussian S_2m's first m rows are sqrt(1/2) S_m, and
    the SRHT's 2m rows contain the m rows of S_m with the same signs (each S_m
    is still a sketch of its kind; the draws are no longer independent across
    levels, a departure from redrawing S at every doubling)."""
    A = np.asarray(A, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    if dual_b is not None:
        dual_b = np.asarray(dual_b, dtype=np.float64)
        b = np.zeros(A.shape[0])
    n, d = A.shape
    if m_init < 1 or (m_init & (m_init - 1)):
        raise ValueError("m_init must be a power of two")
    prm = P.ihs_params(kind, rho, eta)
    m_cap = next_pow2(n) if kind == "srht" else n
    sketch_fn = sketch_fn or SK.sketch
    x_prev = np.zeros(d) if x0 is None else np.asarray(x0, dtype=np.float64).copy()
    x = np.zeros(d) if x1 is None else np.asarray(x1, dtype=np.float64).copy()

    m = m_init
    level = int(round(math.log2(m)))
    passes = 0

    def grad_at(v):
        nonlocal passes
        passes += 1
        if grad_fn is not None:
            return grad_fn(v)
        Av = A @ v
        g = A.T @ (Av - b) + nu * nu * v
        if dual_b is not None:
            g = g - dual_b
        return g, float(Av @ Av)

    draw = (lambda lv: 0) if nested else (lambda lv: lv)
    # Draw S, form SA and cache the factor of H_S.
    fac = linalg.WoodburyFactor(sketch_fn(A, m, kind, seed, draw(level)), nu)
    levels = [m]
    # Initial gradient, preconditioned gradient and decrement r_1.
    g, ax2 = grad_at(x)
    gt = fac.apply(g)
    r = 0.5 * g @ gt
    r1 = r
    trace = []
    history = [(1, x.copy(), fac.SA)] if keep_history else []
    status = "maxiter"
    t = 1
    while t < max_iter:
        scale = tol * math.sqrt(ax2 + nu * nu * (x @ x))
        if r <= 0.0 or math.sqrt(2.0 * prm.Lam * r) <= scale:
            status = "converged"
            # the stopping test's value sqrt(2 Lambda r_t) / (tol ||Abar x_t||), <= 1
            trace.append(("stop", t, m, math.sqrt(2.0 * prm.Lam * max(r, 0.0)) / scale if scale > 0 else 0.0))
            break
        accepted = False
        if variant == "polyak":
            # Polyak candidate, tested by (r_p^+ / r_1)^(1/t).
            xp = x - prm.mu_p * gt + prm.beta_p * (x - x_prev)
            gp, ax2p = grad_at(xp)
            gtp = fac.apply(gp)
            rp = 0.5 * gp @ gtp
            ratio = (rp / r1) ** (1.0 / t) if rp > 0 else 0.0
            if ratio <= prm.c_p:
                trace.append(("polyak", t, m, ratio))
                x_prev, x, g, gt, r, ax2 = x, xp, gp, gtp, rp, ax2p
                accepted = True
            else:
                trace.append(("polyak_reject", t, m, ratio))
        if not accepted:
            # Gradient-IHS candidate, tested by r_gd^+ / r_t.
            xg = x - prm.mu_gd * gt
            gg, ax2g = grad_at(xg)
            gtg = fac.apply(gg)
            rg = 0.5 * gg @ gtg
            ratio = rg / r
            if ratio <= prm.c_gd or m >= m_cap:
                trace.append(("gd" if ratio <= prm.c_gd else "gd_at_cap", t, m, ratio))
                x_prev, x, g, gt, r, ax2 = x, xg, gg, gtg, rg, ax2g
                accepted = True
            elif floor > 0.0 and r <= floor * floor * r1:
                status = "floor"
                trace.append(("floor", t, m, ratio))
                break
            else:
                # Neither candidate improved enough: double m, redraw S,
                # recompute gt_t and r_t, retry the same t.
                trace.append(("double", t, m, ratio))
                m = min(2 * m, m_cap)
                level += 1
                fac = linalg.WoodburyFactor(sketch_fn(A, m, kind, seed, draw(level)), nu)
                levels.append(m)
                gt = fac.apply(g)
                r = 0.5 * g @ gt
                continue
        t += 1
        if keep_history:
            history.append((t, x.copy(), fac.SA))
    return IHSResult(x=x, m=m, level=level, iterations=t, status=status, trace=trace,
                     levels=levels, grad_passes=passes, r=r, r1=r1, history=history)


def adaptive_ihs_dual(A, b, nu, **kw):
    """The underdetermined case (App. A.2): for A of shape (n, d), n <= d, run the
    method on the dual z* = argmin 1/2 ||A^T z||^2 + nu^2/2 ||z||^2 - b^T z, whose
    data matrix is A^T (d x n, overdetermined) and whose gradient is
    A A^T z - b + nu^2 z (App. A.2 drops nu^2 z; the dual objective has it),
    then map back with x = A^T z.  Returns (x, dual result)."""
    A = np.asarray(A, dtype=np.float64)
    res = adaptive_ihs(A.T, np.zeros(A.shape[1]), nu, dual_b=b, **kw)
    return A.T @ res.x, res
