"""Oracle LP data: domain partition, normalisation, residuals and metrics (FP64).

Test infrastructure only (like the whole oracle package): never imported by the product path.

Domain partition (Sec. 2.2, Fig. 2):
  gel  = {f_T != 0}
  band = non-gel voxels with K f_T != 0, or (reading, following the band width
         of Secs. 3.2-3.4) within Euclidean distance <= W of a gel voxel;
         W < 0 means band-free: every non-gel voxel is band.  Everything
         outside the vial cylinder is exterior.
  ext  = the rest.
  active rays = {[P f_T]_j != 0} (unblurred P, with attenuation), mask = rest.

The LP after the Charnes-Cooper transform (Eqs. 19-24), and its two practical
cases (Case 1: Eqs. 32-37 with Eqs. 29-31; Case 2: Eqs. 40-45 with Eq. 39), are
written as  min c^T x  s.t.  G x <= h  over x = (y, u~, v~) with rows

  band (up) rows:  d_i - u~          <= 0      (general, Case 1)
                   d_i               <= 1      (Case 2)
  gel  (up) rows:  d_i - v~ f~_T,i   <= 0      (general, Case 2)
                   d_i               <= f~_U,i (Case 1)
  gel  (lo) rows: -d_i               <= -L_i   (L = f~_T, or f~_L in Case 1)

with d = A^T y, y >= 0 on active rays and y = 0 on masked rays.  The implied
bounds u~ >= 0 and v~ >= 1 are added (they cannot cut the optimum: A^T y >= 0
and f~_T <= A^T y <= v~ f~_T on gel).

Normalisation: general f_crit = min_gel f_T (Sec. 2.5); Case 1 f_L = (1-dl) f_T,
f_U = (1+du) f_T, or explicit per-voxel f_L, f_U (the response-domain bounds
M^-1(m_L), M^-1(m_U) of Sec. 2.7.1), f_crit = min_gel f_L (Eq. 30); Case 2
f_crit = ratio * min_gel f_T (reading of the inhibition threshold).
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np
from scipy import ndimage

from .operators import Geometry, Operators, apply_psf, has_psf

GENERAL, CASE1, CASE2 = 0, 1, 2


@dataclass
class CaseParams:
    case: int = GENERAL
    w1: float = 1.0
    w2: float = 1.0
    tol_lo: float = 0.05        # Case 1: f_L = (1 - tol_lo) f_T
    tol_hi: float = 0.05        # Case 1: f_U = (1 + tol_hi) f_T
    inhibit_ratio: float = 0.8  # Case 2: f_crit = ratio * min_gel f_T
    band_width: int = 10        # voxels; < 0 means band-free
    f_lower: np.ndarray | None = None  # Case 1 with explicit dose bounds f_L, f_U
    f_upper: np.ndarray | None = None  # (e.g. M^-1 of response bounds, Sec. 2.7.1)


EXT, BAND, GEL = 0, 1, 2


def partition(geo: Geometry, f_T: np.ndarray, band_width: int) -> np.ndarray:
    """Region labels per voxel (0 ext, 1 band, 2 gel), array shaped like f_T."""
    f_T = np.asarray(f_T, dtype=np.float64)
    gel = f_T != 0
    ny, nx, nz = f_T.shape
    if geo.vial_radius > 0:
        ys = np.arange(ny) - (ny - 1) / 2.0
        xs = np.arange(nx) - (nx - 1) / 2.0
        Y, X = np.meshgrid(ys, xs, indexing="ij")
        in_vial = (X * X + Y * Y <= geo.vial_radius ** 2)[:, :, None]
        in_vial = np.broadcast_to(in_vial, f_T.shape)
    else:
        in_vial = np.ones(f_T.shape, dtype=bool)
    if band_width < 0:
        band = ~gel
    else:
        if gel.any():
            dist = ndimage.distance_transform_edt(~gel)
            band = (~gel) & (dist <= band_width)
        else:
            band = np.zeros_like(gel)
        if has_psf(geo):
            band |= (~gel) & (apply_psf(geo, gel.astype(np.float64)) > 0)
    band &= in_vial
    lab = np.zeros(f_T.shape, dtype=np.uint8)
    lab[band] = BAND
    lab[gel] = GEL
    return lab


@dataclass
class LPData:
    case: int
    labels: np.ndarray        # (V,) uint8, [y][x][z] order
    ft: np.ndarray            # (V,) normalised target f~_T on gel (general/C2) or f~_L (C1)
    lower: np.ndarray         # (V,) L_i on gel
    upper: np.ndarray         # (V,) constant upper bound on gel (C1: f~_U), else 0
    active: np.ndarray        # (S,) bool
    f_crit: float
    f_T: np.ndarray           # (V,) un-normalised target
    c_u: float
    c_v: float

    @property
    def has_u(self):
        return self.case in (GENERAL, CASE1)

    @property
    def has_v(self):
        return self.case in (GENERAL, CASE2)

    @property
    def gel(self):
        return self.labels == GEL

    @property
    def band(self):
        return self.labels == BAND

    def band_rhs(self):
        """b on band rows: 0 when u~ is a variable, 1 in Case 2."""
        return 0.0 if self.has_u else 1.0

    def h_norm(self) -> float:
        gel, band = self.gel, self.band
        s = band.sum() * self.band_rhs() ** 2
        s += np.sum(self.upper[gel] ** 2) + np.sum(self.lower[gel] ** 2)
        return float(np.sqrt(s))

    def c_norm(self) -> float:
        return float(np.sqrt((self.c_u ** 2 if self.has_u else 0.0)
                             + (self.c_v ** 2 if self.has_v else 0.0)))


def active_rays(ops: Operators, f_T: np.ndarray) -> np.ndarray:
    """Pi^act = {[P f_T]_j != 0} with the unblurred, attenuated P (Sec. 2.2)."""
    return ops.project_raw(f_T).ravel() > 0


def build_lp(geo: Geometry, f_T: np.ndarray, cp: CaseParams,
             precision="f64") -> tuple[LPData, Operators]:
    ops = Operators(geo, precision)
    f_T = np.asarray(f_T, dtype=np.float64)
    lab = partition(geo, f_T, cp.band_width).ravel()
    fT = f_T.ravel()
    gel = lab == GEL
    if not gel.any():
        raise ValueError("empty gelation region")
    V = fT.size
    ft = np.zeros(V)
    lower = np.zeros(V)
    upper = np.zeros(V)
    if cp.case == GENERAL:
        f_crit = fT[gel].min()
        ft[gel] = fT[gel] / f_crit
        lower[gel] = ft[gel]
        c_u, c_v = cp.w1, cp.w2
    elif cp.case == CASE1:
        if cp.f_lower is not None:
            fL = np.asarray(cp.f_lower, dtype=np.float64).ravel()
            fU = np.asarray(cp.f_upper, dtype=np.float64).ravel()
            if not (np.all(fL[gel] > 0) and np.all(fU[gel] >= fL[gel])):
                raise ValueError("explicit bounds need 0 < f_L <= f_U on gel")
        else:
            fL = (1.0 - cp.tol_lo) * fT
            fU = (1.0 + cp.tol_hi) * fT
        f_crit = fL[gel].min()
        ft[gel] = fL[gel] / f_crit
        lower[gel] = ft[gel]
        upper[gel] = fU[gel] / f_crit
        c_u, c_v = 1.0, 0.0
    elif cp.case == CASE2:
        f_crit = cp.inhibit_ratio * fT[gel].min()
        ft[gel] = fT[gel] / f_crit
        lower[gel] = ft[gel]
        c_u, c_v = 0.0, 1.0
    else:
        raise ValueError(cp.case)
    act = active_rays(ops, f_T)
    lp = LPData(cp.case, lab.astype(np.uint8), ft, lower, upper, act,
                float(f_crit), fT, c_u, c_v)
    if lp.has_u and c_u != 0.0 and not lp.band.any():
        # u~ is the band maximum (Eqs. 20, 33): with no band row it is bound by
        # nothing and the LP (free u~, Eqs. 9-24) is unbounded
        raise ValueError("empty band: the band maximum u~ is in no row")
    return lp, ops


def up_bound(lp: LPData, u: float, v: float) -> np.ndarray:
    """Right side U_i of the up rows at scalars (u~, v~): d_i <= U_i (band & gel)."""
    U = np.zeros(lp.labels.size)
    band, gel = lp.band, lp.gel
    U[band] = u if lp.has_u else 1.0
    U[gel] = v * lp.ft[gel] if lp.has_v else lp.upper[gel]
    return U


def kkt(lp: LPData, d, g, u, v, lam_up, lam_lo) -> dict:
    """Residuals, objectives and the relative KKT error of a primal-dual point.

    d = A^T y (primal), g = A (lam_up - lam_lo) (dual, Eq. 51).  Stationarity
    for the scalars (Eqs. 48-49) with the implied bounds u~ >= 0, v~ >= 1 gives
    reduced costs r_u = c_u - sum_band lam_up, r_v = c_v - sum_gel f~ lam_up;
    their negative parts are dual residuals and v~'s lower bound adds
    1 * max(r_v, 0) to the dual objective.  On active rays the reduced cost of
    y >= 0 is g (its negative part is the residual).
    """
    band, gel = lp.band, lp.gel
    d = np.asarray(d, dtype=np.float64).ravel()
    g = np.asarray(g, dtype=np.float64).ravel()
    lam_up = np.asarray(lam_up, dtype=np.float64).ravel()
    lam_lo = np.asarray(lam_lo, dtype=np.float64).ravel()
    U = up_bound(lp, u, v)
    rp2 = np.sum(np.maximum(d[band] - U[band], 0.0) ** 2)
    rp2 += np.sum(np.maximum(d[gel] - U[gel], 0.0) ** 2)
    rp2 += np.sum(np.maximum(lp.lower[gel] - d[gel], 0.0) ** 2)
    rd2 = np.sum(np.minimum(g[lp.active], 0.0) ** 2)
    S_band = lam_up[band].sum()
    S_gel = np.sum(lp.ft[gel] * lam_up[gel])
    pobj = 0.0
    dobj = np.sum(lp.lower[gel] * lam_lo[gel])
    if lp.has_u:
        r_u = lp.c_u - S_band
        rd2 += min(r_u, 0.0) ** 2
        pobj += lp.c_u * u
    else:
        dobj -= lp.band_rhs() * S_band
    if lp.has_v:
        r_v = lp.c_v - S_gel
        rd2 += min(r_v, 0.0) ** 2
        dobj += max(r_v, 0.0)
        pobj += lp.c_v * v
    else:
        dobj -= np.sum(lp.upper[gel] * lam_up[gel])
    rp, rd = float(np.sqrt(rp2)), float(np.sqrt(rd2))
    rel_p = rp / (1.0 + lp.h_norm())
    rel_d = rd / (1.0 + lp.c_norm())
    gap = abs(pobj - dobj)
    rel_gap = gap / (1.0 + abs(pobj) + abs(dobj))
    return dict(r_primal=rp, r_dual=rd, pobj=float(pobj), dobj=float(dobj),
                gap=float(gap), rel_primal=rel_p, rel_dual=rel_d,
                rel_gap=rel_gap, kkt=max(rel_p, rel_d, rel_gap),
                S_band=float(S_band), S_gel=float(S_gel))


def metrics(lp: LPData, d) -> dict:
    """Scale-invariant metrics of a dose field d = A^T y.

    DTVR and DSR in the normalised form of Eq. 8 (with f~_T = f_T / f_crit),
    PSR_f of Eq. 46, the dose-domain post-scaling factor of Eq. 27 with unit
    weights (alpha* = <f~*, f_T>_gel / <f~*, f~*>_gel), and the recovered
    Charnes-Cooper scale s = min_gel(d / f~) of the LP's own lower-bound
    profile (t = 1/s, Eq. 18; s = 1 at an optimum).
    """
    d = np.asarray(d, dtype=np.float64).ravel()
    gel, band = lp.gel, lp.band
    fT = lp.f_T
    ftil = fT / lp.f_crit
    r = d[gel] / ftil[gel]
    out = dict(dtvr_f=float(r.max() / r.min()) if r.min() > 0 else float("inf"))
    band_max = float(d[band].max()) if band.any() else 0.0
    out["dsr"] = band_max / float(r.min()) if r.min() > 0 else float("inf")
    gel_min = float(d[gel].min())
    out["psr_f"] = gel_min / band_max if band_max > 0 else float("inf")
    num = float(np.dot(d[gel], fT[gel]))
    den = float(np.dot(d[gel], d[gel]))
    out["alpha"] = num / den if den > 0 else 0.0
    s = float((d[gel] / lp.lower[gel]).min())
    out["s"] = s
    out["band_max"] = band_max
    out["gel_max_ratio"] = float((d[gel] / lp.ft[gel]).max())
    return out
