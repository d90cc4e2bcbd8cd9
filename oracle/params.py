"""Algorithmic parameters of the gradient- and Polyak-IHS.

Thm 2.1: mu_gd(l, L) = 2 / (1/l + 1/L),  c_gd(l, L) = ((L - l) / (L + l))^2.
Thm 2.2: mu_p(l, L) = 4 / (1/sqrt(l) + 1/sqrt(L))^2,
         beta_p(l, L) = c_p(l, L) = ((sqrt(L) - sqrt(l)) / (sqrt(L) + sqrt(l)))^2.
Def 3.1 (Gaussian): c_eta = (1 + 3 sqrt(eta))^2, l = (1 - sqrt(c_eta rho))^2,
         L = (1 + sqrt(c_eta rho))^2, for rho <= 0.18, eta <= 0.01 (Thm 3.1).
Def 3.2 (SRHT): l = 1 - sqrt(rho), L = 1 + sqrt(rho), rho in (0, 1).
Thm 4.1 / 4.2 run Algorithm 1 with cbar_gd = c_gd and cbar_p = c_p.
"""
import math
from dataclasses import dataclass


def mu_gd(lo, hi):
    return 2.0 / (1.0 / lo + 1.0 / hi)


def c_gd(lo, hi):
    return ((hi - lo) / (hi + lo)) ** 2


def mu_p(lo, hi):
    return 4.0 / (1.0 / math.sqrt(lo) + 1.0 / math.sqrt(hi)) ** 2


def beta_p(lo, hi):
    return ((math.sqrt(hi) - math.sqrt(lo)) / (math.sqrt(hi) + math.sqrt(lo))) ** 2


c_p = beta_p


def bounds_gaussian(rho, eta):
    """(lambda_{rho,eta}, Lambda_{rho,eta}) of Def 3.1."""
    if not (0 < rho <= 0.18 and 0 < eta <= 0.01):
        raise ValueError("Def 3.1 needs rho in (0, 0.18], eta in (0, 0.01]")
    c_eta = (1.0 + 3.0 * math.sqrt(eta)) ** 2
    s = math.sqrt(c_eta * rho)
    return (1.0 - s) ** 2, (1.0 + s) ** 2


def bounds_srht(rho):
    """(lambda_rho, Lambda_rho) of Def 3.2."""
    if not 0 < rho < 1:
        raise ValueError("Def 3.2 needs rho in (0, 1)")
    s = math.sqrt(rho)
    return 1.0 - s, 1.0 + s


@dataclass(frozen=True)
class IHSParams:
    lam: float
    Lam: float
    mu_gd: float
    c_gd: float
    mu_p: float
    beta_p: float
    c_p: float


def ihs_params(kind, rho=0.1, eta=0.01):
    """Parameters Thm 4.1 (Gaussian) / Thm 4.2 (SRHT) prescribe."""
    lo, hi = bounds_gaussian(rho, eta) if kind == "gauss" else bounds_srht(rho)
    return IHSParams(lo, hi, mu_gd(lo, hi), c_gd(lo, hi), mu_p(lo, hi), beta_p(lo, hi), c_p(lo, hi))


def srht_oversampling(n, de):
    """C(n, d_e) = 16/3 (1 + sqrt(8 log(d_e n) / d_e))^2 (Sec. 3.2)."""
    return 16.0 / 3.0 * (1.0 + math.sqrt(8.0 * math.log(de * n) / de)) ** 2


def sketch_size_bound(kind, de, rho, n=None, c0=5.0):
    """Upper bound on the adaptive sketch size: 2 c0 d_e / rho (Thm 4.1) or
    2 a_rho C(n, d_e) d_e log d_e / rho (Thm 4.2)."""
    if kind == "gauss":
        return 2.0 * c0 * de / rho
    a_rho = (1 + math.sqrt(rho)) / (1 - math.sqrt(rho))
    return 2.0 * a_rho * srht_oversampling(n, de) * de * math.log(de) / rho


def rejected_steps_bound(kind, de, rho, m_init=1, n=None, c0=5.0):
    """Bound on the number K of rejected updates (Thm 4.1 / Thm 4.2)."""
    if kind == "gauss":
        return math.log(c0 * de / (m_init * rho)) / math.log(2.0) + 1.0
    a_rho = (1 + math.sqrt(rho)) / (1 - math.sqrt(rho))
    return math.log(a_rho * srht_oversampling(n, de) * de * math.log(de) / (m_init * rho)) / math.log(2.0) + 1.0
