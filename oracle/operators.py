"""Oracle forward model: P^T, P, attenuation and the PSF K (FP64, CPU).

Test infrastructure only (like the whole oracle package): never imported by the product path.

Forward model (Sec. 2.3, Eqs. 2-3): the dose is f = A^T g with A^T = K P^T,
where P^T backprojects a sinogram g into object space and K is the object-space
PSF.  P is the adjoint of P^T (Sec. 2.3), and A = P K^T = P K (K symmetric).

The paper fixes no discretisation; the readings used here are:

* Voxel centres x = ix - (nx-1)/2, y = iy - (ny-1)/2 (unit spacing); z is the
  rotation axis and the operator acts on every z-slice alike (slice-separable).
* Angle theta_k, detector coordinate u = x cos(theta) + y sin(theta) + (nu-1)/2.
  P^T is pixel-driven linear interpolation: with i0 = floor(u), w = u - i0 the
  voxel receives (1-w) g[k, i0] + w g[k, i0+1]; taps outside [0, nu-1] are 0.
* P is defined as the exact transpose of that matrix (built here explicitly).
* Beer-Lambert attenuation (only with a vial of radius R > 0): light enters the
  vial at depth -sqrt(R^2 - s^2) and travels along d = (-sin, cos); the depth
  of the voxel is t = -x sin + y cos.  The tap to bin j is weighted by
  exp(-mu (t + sqrt(R^2 - s_j^2))) with s_j = j - (nu-1)/2 the bin-centre
  offset, and 0 when |s_j| > R.  Voxels with x^2 + y^2 > R^2 are outside the
  vial and take no part in the operator.
* PSF: separable Gaussian, taps exp(-i^2/(2 sigma^2)) normalised to sum 1 on
  i in [-R_a, R_a] per axis, zero padding (so K^T = K); sigma_a = 0 means the
  identity on that axis.

Data layout: volumes [ny][nx][nz], sinograms [n_angles][n_det][nz] (z fastest).
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np
import scipy.sparse as sp


@dataclass
class Geometry:
    nx: int
    ny: int
    nz: int
    angles: np.ndarray          # float64, radians
    n_det: int
    vial_radius: float = 0.0    # <= 0: no vial (then mu must be 0)
    mu: float = 0.0             # attenuation per voxel length
    psf_sigma: tuple = (0.0, 0.0, 0.0)   # (sigma_x, sigma_y, sigma_z)
    psf_trunc: float = 4.0

    @property
    def n_angles(self) -> int:
        return len(self.angles)

    @property
    def vol_shape(self):
        return (self.ny, self.nx, self.nz)

    @property
    def sino_shape(self):
        return (self.n_angles, self.n_det, self.nz)

    def psf_radii(self):
        """R_a = ceil(trunc * sigma_a) per axis (x, y, z); 0 where sigma_a = 0."""
        return tuple(int(math.ceil(self.psf_trunc * s)) if s > 0 else 0
                     for s in self.psf_sigma)


def _f32(a):
    return np.asarray(a, dtype=np.float32)


def detector_coordinate(x, y, cos_t, sin_t, off, precision="f64"):
    """u = x cos + y sin + off in the requested arithmetic.

    "f64": IEEE double, evaluated as (x*cos) + ((y*sin) + off).
    "f32": single precision with two fused multiply-adds,
           u = fma(x, cos, fma(y, sin, off)), cos/sin/off rounded to float32.
           Each fma is emulated exactly: the float64 value of a*b + c is exact
           for these operand ranges (|x|,|y| < 2^12 half-integers, 24-bit
           cos/sin), so one rounding to float32 reproduces the fused result.
    The "f32" mode exists so that integer decisions that depend on u (which
    rays are active) can be compared with the single-precision kernels in the
    same precision; values are always accumulated in FP64 here.
    """
    if precision == "f64":
        return x * cos_t + (y * sin_t + off)
    if precision == "f32":
        c32 = np.float64(_f32(cos_t))
        s32 = np.float64(_f32(sin_t))
        o32 = np.float64(_f32(off))
        inner = _f32(np.asarray(y, np.float64) * s32 + o32).astype(np.float64)
        return _f32(np.asarray(x, np.float64) * c32 + inner).astype(np.float64)
    raise ValueError(precision)


def backprojector_matrix(geo: Geometry, precision="f64", with_attenuation=True):
    """The 2-D slice operator P^T (or P_mu^T) as a sparse (nx*ny, n_angles*n_det) matrix.

    Row index iy*nx + ix (voxel), column index k*n_det + j (ray).  Entries are
    the interpolation weights times the Beer-Lambert factor of that tap.
    """
    nx, ny, nu = geo.nx, geo.ny, geo.n_det
    off = (nu - 1) / 2.0
    xs = np.arange(nx) - (nx - 1) / 2.0
    ys = np.arange(ny) - (ny - 1) / 2.0
    Y, X = np.meshgrid(ys, xs, indexing="ij")
    X = X.ravel()
    Y = Y.ravel()
    vox = np.arange(nx * ny)
    R = geo.vial_radius
    if R > 0:
        inside = X * X + Y * Y <= R * R
    else:
        if geo.mu != 0.0:
            raise ValueError("attenuation needs a vial radius")
        inside = np.ones_like(X, dtype=bool)
    X, Y, vox = X[inside], Y[inside], vox[inside]
    rows, cols, vals = [], [], []
    for k, th in enumerate(np.asarray(geo.angles, dtype=np.float64)):
        c, s = math.cos(th), math.sin(th)
        u = detector_coordinate(X, Y, c, s, off, precision)
        i0 = np.floor(u)
        w = u - i0
        i0 = i0.astype(np.int64)
        t = -X * s + Y * c
        for j, wt in ((i0, 1.0 - w), (i0 + 1, w)):
            ok = (j >= 0) & (j < nu) & (wt > 0)
            jj = j[ok]
            val = wt[ok]
            if R > 0:
                sj = jj - off
                in_vial = np.abs(sj) <= R
                path = t[ok] + np.sqrt(np.maximum(R * R - sj * sj, 0.0))
                att = np.exp(-geo.mu * path) if with_attenuation else 1.0
                val = np.where(in_vial, val * att, 0.0)
                keep = val > 0
                jj, val, vv = jj[keep], val[keep], vox[ok][keep]
            else:
                vv = vox[ok]
            rows.append(vv)
            cols.append(k * nu + jj)
            vals.append(val)
    rows = np.concatenate(rows)
    cols = np.concatenate(cols)
    vals = np.concatenate(vals)
    return sp.csr_matrix((vals, (rows, cols)), shape=(nx * ny, geo.n_angles * nu))


def psf_taps(sigma: float, radius: int) -> np.ndarray:
    """Normalised Gaussian taps k[i], i = -radius..radius (identity when sigma = 0)."""
    if sigma <= 0 or radius == 0:
        return np.ones(1)
    i = np.arange(-radius, radius + 1, dtype=np.float64)
    e = np.exp(-(i * i) / (2.0 * sigma * sigma))
    return e / e.sum()


def psf_tap_derivative(sigma: float, radius: int) -> np.ndarray:
    """d k[i] / d sigma for the normalised taps (quotient rule, radius frozen)."""
    if sigma <= 0 or radius == 0:
        return np.zeros(1)
    i = np.arange(-radius, radius + 1, dtype=np.float64)
    e = np.exp(-(i * i) / (2.0 * sigma * sigma))
    de = e * (i * i) / sigma ** 3
    S, dS = e.sum(), de.sum()
    return (de * S - e * dS) / (S * S)


def convolve_axis(vol: np.ndarray, taps: np.ndarray, axis: int) -> np.ndarray:
    """out[i] = sum_m taps[m] * vol[i + m - R] along `axis`, zero outside the grid."""
    R = (len(taps) - 1) // 2
    if R == 0:
        return vol * taps[0]
    n = vol.shape[axis]
    pad = [(0, 0)] * vol.ndim
    pad[axis] = (R, R)
    p = np.pad(vol, pad)
    out = np.zeros_like(vol, dtype=np.float64)
    for m in range(2 * R + 1):
        sl = [slice(None)] * vol.ndim
        sl[axis] = slice(m, m + n)
        out += taps[m] * p[tuple(sl)]
    return out


def apply_psf(geo: Geometry, vol: np.ndarray, sigma=None, radii=None,
              deriv_axis: int | None = None) -> np.ndarray:
    """K vol (or dK/dsigma_a vol with deriv_axis = a in {0:x, 1:y, 2:z}).

    Volume axes are (y, x, z); sigma is ordered (x, y, z).
    """
    sigma = geo.psf_sigma if sigma is None else sigma
    radii = geo.psf_radii() if radii is None else radii
    out = np.asarray(vol, dtype=np.float64)
    axis_of = {0: 1, 1: 0, 2: 2}      # sigma index -> array axis
    for a in range(3):
        if deriv_axis == a:
            taps = psf_tap_derivative(sigma[a], radii[a])
        else:
            taps = psf_taps(sigma[a], radii[a])
        out = convolve_axis(out, taps, axis_of[a])
    return out


def has_psf(geo: Geometry) -> bool:
    return any(s > 0 for s in geo.psf_sigma)


class Operators:
    """A^T = K P_mu^T and A = P_mu K for one geometry (FP64, explicit matrices)."""

    def __init__(self, geo: Geometry, precision="f64"):
        self.geo = geo
        self.PT = backprojector_matrix(geo, precision)   # (V2, S2)
        self.P = self.PT.T.tocsr()                       # exact transpose

    def _vol2(self, v):
        g = self.geo
        return np.asarray(v, dtype=np.float64).reshape(g.ny * g.nx, g.nz)

    def _sino2(self, s):
        g = self.geo
        return np.asarray(s, dtype=np.float64).reshape(g.n_angles * g.n_det, g.nz)

    def backproject_raw(self, sino):
        """P_mu^T sino (no PSF), volume [ny][nx][nz]."""
        g = self.geo
        return (self.PT @ self._sino2(sino)).reshape(g.vol_shape)

    def project_raw(self, vol):
        """P_mu vol (no PSF), sinogram [n_angles][n_det][nz]."""
        g = self.geo
        return (self.P @ self._vol2(vol)).reshape(g.sino_shape)

    def AT(self, sino):
        """A^T sino = K P_mu^T sino (Eq. 3)."""
        b = self.backproject_raw(sino)
        return apply_psf(self.geo, b) if has_psf(self.geo) else b

    def A(self, vol):
        """A vol = P_mu K vol (adjoint of A^T; K is symmetric)."""
        v = apply_psf(self.geo, vol) if has_psf(self.geo) else np.asarray(vol, np.float64)
        return self.project_raw(v)
