"""Single-output evaluation of the oracle operators at full size (FP64).

Test infrastructure only (like the whole oracle package): never imported by the product path.

At 256^3 x 360 views the explicit matrices are too large for quick tests, but
any one output of P^T, P or K is a short sum that follows directly from the
definitions in `operators` (Sec. 2.3, Eqs. 2-3): these functions compute that
sum for one voxel or one ray so that sampled outputs of a full-size GPU launch
can be checked one by one.
"""
from __future__ import annotations

import math

import numpy as np

from .operators import Geometry, psf_taps


def _tap_weight(geo: Geometry, x, y, c, s, j):
    """Attenuation factor of the tap from voxel (x, y) to bin j (1 without a vial)."""
    R = geo.vial_radius
    if R <= 0:
        return np.ones_like(np.asarray(j, dtype=np.float64))
    off = (geo.n_det - 1) / 2.0
    sj = np.asarray(j, dtype=np.float64) - off
    t = -x * s + y * c
    path = t + np.sqrt(np.maximum(R * R - sj * sj, 0.0))
    return np.where(np.abs(sj) <= R, np.exp(-geo.mu * path), 0.0)


def backproject_voxel(geo: Geometry, sino: np.ndarray, iy: int, ix: int, iz: int) -> float:
    """[P_mu^T sino] at voxel (iy, ix, iz): sum over angles of the two taps."""
    x = ix - (geo.nx - 1) / 2.0
    y = iy - (geo.ny - 1) / 2.0
    R = geo.vial_radius
    if R > 0 and x * x + y * y > R * R:
        return 0.0
    off = (geo.n_det - 1) / 2.0
    total = 0.0
    for k, th in enumerate(geo.angles):
        c, s = math.cos(th), math.sin(th)
        u = x * c + (y * s + off)
        i0 = math.floor(u)
        w = u - i0
        for j, wt in ((i0, 1.0 - w), (i0 + 1, w)):
            if 0 <= j < geo.n_det and wt > 0:
                total += wt * float(_tap_weight(geo, x, y, c, s, j)) * float(sino[k, j, iz])
    return total


def project_ray(geo: Geometry, vol: np.ndarray, k: int, j: int, iz: int) -> float:
    """[P_mu vol] at ray (k, j, iz): sum over all voxels whose taps reach bin j."""
    xs = np.arange(geo.nx) - (geo.nx - 1) / 2.0
    ys = np.arange(geo.ny) - (geo.ny - 1) / 2.0
    Y, X = np.meshgrid(ys, xs, indexing="ij")
    th = geo.angles[k]
    c, s = math.cos(th), math.sin(th)
    off = (geo.n_det - 1) / 2.0
    u = X * c + (Y * s + off)
    i0 = np.floor(u)
    w = u - i0
    wt = np.where(i0 == j, 1.0 - w, 0.0) + np.where(i0 + 1 == j, w, 0.0)
    R = geo.vial_radius
    if R > 0:
        wt = np.where(X * X + Y * Y <= R * R, wt, 0.0)
    wt = wt * _tap_weight(geo, X, Y, c, s, j)
    return float(np.sum(wt * vol[:, :, iz]))


def psf_voxel(geo: Geometry, vol: np.ndarray, iy: int, ix: int, iz: int,
              sigma=None, radii=None) -> float:
    """[K vol] at one voxel: the separable taps summed over the box neighbourhood."""
    sigma = geo.psf_sigma if sigma is None else sigma
    radii = geo.psf_radii() if radii is None else radii
    kx = psf_taps(sigma[0], radii[0])
    ky = psf_taps(sigma[1], radii[1])
    kz = psf_taps(sigma[2], radii[2])
    Rx, Ry, Rz = (len(kx) - 1) // 2, (len(ky) - 1) // 2, (len(kz) - 1) // 2
    total = 0.0
    ny, nx, nz = vol.shape
    for a in range(-Ry, Ry + 1):
        yy = iy + a
        if not 0 <= yy < ny:
            continue
        for b in range(-Rx, Rx + 1):
            xx = ix + b
            if not 0 <= xx < nx:
                continue
            lo, hi = max(0, iz - Rz), min(nz, iz + Rz + 1)
            seg = vol[yy, xx, lo:hi].astype(np.float64)
            taps = kz[(lo - iz + Rz):(hi - iz + Rz)]
            total += ky[a + Ry] * kx[b + Rx] * float(seg @ taps)
    return total
