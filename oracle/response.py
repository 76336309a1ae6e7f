"""Oracle material response (Sec. 2.1; Eqs. 4-5, 28, 46), plain FP64 numpy.

Test infrastructure only (like the whole oracle package): never imported by the product path.

The resin's response to dose is Richards' generalised logistic curve
(Eq. 4) with lower and upper asymptotes alpha < k, growth rate beta > 0,
shape gamma > 0 and location f0; its closed-form inverse (Eq. 5) turns a
target response m_T into the target dose f_T, and the response tolerances
m_L = (1 - eps_L) m_T, m_U = (1 + eps_U) m_T of Case 1 into dose bounds
f_L, f_U (Sec. 2.7.1).  After the solve, the post-scaling factor alpha may be
chosen in the response domain by minimising Phi_m (Eq. 28, unit weights),
and the separation PSR_m (Eq. 46) and the uniformity DTVR_m (the response
analogue of Eq. 6) read the scaled dose through M.

The paper prints no resin constants; every function takes them as input.
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np
from scipy.optimize import minimize_scalar

from .lp import LPData


@dataclass(frozen=True)
class Richards:
    alpha: float
    k: float
    beta: float
    gamma: float
    f0: float


def response(p: Richards, f):
    """m = M(f) = alpha + (k - alpha) / [1 + exp(-beta (f - f0))]^(1/gamma)  (Eq. 4)."""
    f = np.asarray(f, dtype=np.float64)
    with np.errstate(over="ignore"):  # exp -> inf far below f0 gives the asymptote alpha
        return p.alpha + (p.k - p.alpha) / (1.0 + np.exp(-p.beta * (f - p.f0))) ** (1.0 / p.gamma)


def response_inverse(p: Richards, m):
    """f = M^-1(m) = f0 - ln[((k - alpha) / (m - alpha))^gamma - 1] / beta  (Eq. 5)
    for alpha < m < k; m <= alpha (no prescription) gives 0; m >= k is outside
    the invertible range and raises."""
    m = np.asarray(m, dtype=np.float64)
    if np.any(m >= p.k) or np.any(np.isnan(m)):
        raise ValueError("response outside the invertible range")
    out = np.zeros_like(m)
    ok = m > p.alpha
    out[ok] = p.f0 - np.log(((p.k - p.alpha) / (m[ok] - p.alpha)) ** p.gamma - 1.0) / p.beta
    return out


def dose_bounds(p: Richards, m_T, eps_lo: float, eps_hi: float):
    """(f_T, f_L, f_U) = M^-1 of (m_T, (1 - eps_lo) m_T, (1 + eps_hi) m_T) (Eq. 5, Sec. 2.7.1)."""
    m_T = np.asarray(m_T, dtype=np.float64)
    return (response_inverse(p, m_T), response_inverse(p, (1.0 - eps_lo) * m_T),
            response_inverse(p, (1.0 + eps_hi) * m_T))


def phi_m(p: Richards, alpha: float, d, m_T, gel) -> float:
    """Phi_m(alpha) = sum_gel (M(alpha d_i) - m_T,i)^2  (Eq. 28, unit weights)."""
    d = np.asarray(d, dtype=np.float64).ravel()[gel]
    m = np.asarray(m_T, dtype=np.float64).ravel()[gel]
    return float(np.sum((response(p, alpha * d) - m) ** 2))


def alpha_m(p: Richards, d, m_T, gel, centre: float) -> float:
    """argmin over alpha of Phi_m: the best of 4001 geometrically spaced factors
    in [centre / 16, 16 centre], then bounded Brent between its neighbours."""
    grid = centre * np.geomspace(1.0 / 16.0, 16.0, 4001)
    vals = np.array([phi_m(p, a, d, m_T, gel) for a in grid])
    j = int(np.argmin(vals))
    lo, hi = grid[max(j - 1, 0)], grid[min(j + 1, grid.size - 1)]
    res = minimize_scalar(lambda a: phi_m(p, a, d, m_T, gel), bounds=(lo, hi), method="bounded",
                          options=dict(xatol=1e-12 * centre))
    return float(res.x) if res.fun <= vals[j] else float(grid[j])


def response_metrics(p: Richards, lp: LPData, d, m_T, alpha: float) -> dict:
    """PSR_m (Eq. 46), DTVR_m = max_gel(m / m_T) / min_gel(m / m_T) and their
    parts, for the response m = M(alpha d) of the scaled dose."""
    d = np.asarray(d, dtype=np.float64).ravel()
    mT = np.asarray(m_T, dtype=np.float64).ravel()
    gel, band = lp.gel, lp.band
    m = response(p, alpha * d)
    q = m[gel] / mT[gel]
    out = dict(alpha=alpha, phi=phi_m(p, alpha, d, mT, gel), ratio_min=float(q.min()),
               ratio_max=float(q.max()), m_gel_min=float(m[gel].min()),
               m_band_max=float(m[band].max()) if band.any() else 0.0)
    out["dtvr_m"] = out["ratio_max"] / out["ratio_min"]
    out["psr_m"] = out["m_gel_min"] / out["m_band_max"] if band.any() else math.inf
    return out
