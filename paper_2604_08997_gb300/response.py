"""Response-domain front and back end (Sec. 2.1, Eqs. 4-5; Sec. 2.7.1; Eqs. 28, 46).

A target is prescribed as a material response m_T (conversion, refractive
index, ...), related to dose by Richards' curve M (Eq. 4) with the resin's
constants.  The front end maps it to the dose LP through M^-1 (Eq. 5):

- general form and Case 2: f_T = M^-1(m_T); Case 2's inhibition threshold is
  a response m_crit, f_crit = M^-1(m_crit), i.e. the ratio
  f_crit / min_gel f_T = M^-1(m_crit) / M^-1(min_gel m_T) (M is increasing);
- Case 1: response tolerances m_L = (1 - eps_L) m_T, m_U = (1 + eps_U) m_T
  become per-voxel dose bounds f_L = M^-1(m_L), f_U = M^-1(m_U), which are
  not proportional to f_T, so the context is made by sipo_create_bounded.

The back end (`response_metrics`) post-scales the solved dose in the response
domain (Eq. 28) and reports PSR_m (Eq. 46) and DTVR_m.  Every map and
reduction runs in libsipo; torch only holds the device buffers.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np

from ._abi import (SIPO_CASE2, SIPO_GENERAL, sipo_create, sipo_create_bounded, sipo_response_inhibit_ratio,
                   sipo_response_map, sipo_response_metrics)


@dataclass(frozen=True)
class Richards:
    """Richards' curve (Eq. 4): asymptotes alpha < k, rate beta > 0, shape gamma > 0, location f0."""
    alpha: float
    k: float
    beta: float
    gamma: float
    f0: float

    def as_tuple(self):
        return (self.alpha, self.k, self.beta, self.gamma, self.f0)


def _device(a):
    import torch
    if isinstance(a, np.ndarray):
        a = torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32))
    return a.to(device="cuda", dtype=torch.float32).contiguous()


def response_to_dose(M: Richards, m, scale: float = 1.0):
    """M^-1(scale m) (Eq. 5) as a new float32 CUDA tensor; 0 where scale m <= alpha."""
    import torch
    src = _device(m)
    dst = torch.empty_like(src)
    sipo_response_map(M.as_tuple(), src, dst, inverse=True, scale=scale)
    return dst


def dose_to_response(M: Richards, f, scale: float = 1.0):
    """M(scale f) (Eq. 4) as a new float32 CUDA tensor."""
    import torch
    src = _device(f)
    dst = torch.empty_like(src)
    sipo_response_map(M.as_tuple(), src, dst, inverse=False, scale=scale)
    return dst


def response_case1(geometry: dict, m_T, M: Richards, eps_lo: float = 0.05, eps_hi: float = 0.05,
                   band_width: int = 10, tolerances: dict | None = None):
    """Case 1 with response tolerances: f_L = M^-1((1 - eps_lo) m_T), f_U = M^-1((1 + eps_hi) m_T)."""
    f_T = response_to_dose(M, m_T)
    f_L = response_to_dose(M, m_T, 1.0 - eps_lo)
    f_U = response_to_dose(M, m_T, 1.0 + eps_hi)
    return sipo_create_bounded(geometry, f_T, f_L, f_U, dict(band_width=band_width), tolerances or {})


def response_case2(geometry: dict, m_T, M: Richards, m_crit: float, band_width: int = 10,
                   tolerances: dict | None = None):
    """Case 2 with the inhibition threshold given as a response m_crit (f_crit = M^-1(m_crit))."""
    m = _device(m_T)
    f_T = response_to_dose(M, m)
    ratio, _ = sipo_response_inhibit_ratio(M.as_tuple(), m, m_crit)
    return sipo_create(geometry, f_T, dict(kase=SIPO_CASE2, inhibit_ratio=ratio, band_width=band_width),
                       tolerances or {})


def response_general(geometry: dict, m_T, M: Richards, w1: float = 1.0, w2: float = 1.0,
                     band_width: int = 10, tolerances: dict | None = None):
    """General form on the dose target f_T = M^-1(m_T)."""
    f_T = response_to_dose(M, m_T)
    return sipo_create(geometry, f_T, dict(kase=SIPO_GENERAL, w1=w1, w2=w2, band_width=band_width),
                       tolerances or {})


def response_metrics(ctx, M: Richards, m_T, alpha: float = 0.0) -> dict:
    """Response-domain post-scaling (alpha <= 0: Eq. 28 minimised) and PSR_m / DTVR_m of ctx's last solve."""
    return sipo_response_metrics(ctx, M.as_tuple(), _device(m_T), alpha)
