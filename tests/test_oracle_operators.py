"""Pins for the oracle forward model (CPU only).

Each test checks the oracle against something other than itself: closed forms
(analytic Radon transforms of discs and spheres, with and without Beer-Lambert
attenuation), special angles that reduce to column/row sums, conservation
laws of linear interpolation, a library convolution, exact rational
arithmetic, and finite differences.
"""
import math
from fractions import Fraction

import numpy as np
import pytest
from scipy import ndimage

from oracle.operators import (Geometry, Operators, apply_psf, backprojector_matrix,
                              detector_coordinate, psf_tap_derivative, psf_taps)
from oracle import sample
from synthetic.targets import discs_2d, uniform_angles


def _disc_area(n, r, cx, cy, ss=8):
    """Area-weighted disc occupancy (supersampled ss x ss per voxel)."""
    c = np.arange(n) - (n - 1) / 2
    off = (np.arange(ss) + 0.5) / ss - 0.5
    f = np.zeros((n, n))
    for a in off:
        for b in off:
            Y, X = np.meshgrid(c + a, c + b, indexing="ij")
            f += ((X - cx) ** 2 + (Y - cy) ** 2 <= r * r)
    return f / ss / ss


def test_interpolation_conserves_mass_per_angle():
    """Sum over bins of [P f] at each angle equals sum f (weights 1-w and w sum to 1)."""
    rng = np.random.default_rng(0)
    n, nu = 24, 37          # 24*sqrt(2) + 2 < 37: every tap stays on the detector
    geo = Geometry(n, n, 2, rng.uniform(0, np.pi, 11), nu)
    ops = Operators(geo)
    f = rng.uniform(size=geo.vol_shape)
    p = ops.project_raw(f)
    np.testing.assert_allclose(p.sum(axis=1), np.broadcast_to(f.sum(axis=(0, 1)), (11, 2)),
                               rtol=1e-13)


def test_backprojection_of_ones_counts_angles():
    """P^T 1 = n_angles on every voxel whose taps stay on the detector."""
    rng = np.random.default_rng(1)
    n, nu = 20, 31
    geo = Geometry(n, n, 1, rng.uniform(0, np.pi, 13), nu)
    b = Operators(geo).backproject_raw(np.ones(geo.sino_shape))
    np.testing.assert_allclose(b, 13.0, rtol=1e-13)


def test_axis_angles_reduce_to_column_and_row_sums():
    rng = np.random.default_rng(2)
    # n = n_det: at theta = 0, u = x + (n-1)/2 = ix exactly, so bin ix gets column ix
    n = 16
    geo = Geometry(n, n, 1, np.array([0.0, math.pi / 2]), n)
    f = rng.uniform(size=geo.vol_shape)
    p = Operators(geo).project_raw(f)[:, :, 0]
    np.testing.assert_allclose(p[0], f[:, :, 0].sum(axis=0), rtol=1e-12)
    np.testing.assert_allclose(p[1], f[:, :, 0].sum(axis=1), rtol=1e-12, atol=1e-12)
    # 64^2 grid, 91 bins: u = ix + 13.5, each column splits 1/2 : 1/2 over bins ix+13, ix+14
    geo = Geometry(64, 64, 1, np.array([0.0]), 91)
    f = rng.uniform(size=geo.vol_shape)
    p = Operators(geo).project_raw(f)[0, :, 0]
    col = f[:, :, 0].sum(axis=0)
    expect = np.zeros(91)
    expect[13:77] += 0.5 * col
    expect[14:78] += 0.5 * col
    np.testing.assert_allclose(p, expect, rtol=1e-12)


@pytest.mark.parametrize("n,r,bound", [(64, 14, 0.05), (128, 28, 0.025), (256, 56, 0.013)])
@pytest.mark.parametrize("attenuated", [False, True])
def test_disc_matches_analytic_radon(n, r, bound, attenuated):
    """P of an off-centre area-weighted disc vs the analytic (attenuated) Radon transform.

    Plain: 2 sqrt(r^2 - (s - s0)^2).  Attenuated (vial radius R, depth
    t = -x sin + y cos): exp(-mu sqrt(R^2 - s^2)) exp(-mu t0) 2 sinh(mu a) / mu
    with a = sqrt(r^2 - (s - s0)^2) and t0 the depth of the disc centre.
    The discretisation error falls roughly as 1/r.
    """
    rng = np.random.default_rng(0)
    ang = np.sort(rng.uniform(0, np.pi, 12))
    nu = int(n * 1.45)
    mu = 0.01 * 64 / n if attenuated else 0.0
    geo = Geometry(n, n, 1, ang, nu, vial_radius=0.48 * n, mu=mu)
    cx, cy = 0.07 * n, -0.05 * n
    f = _disc_area(n, r, cx, cy)
    p = Operators(geo).project_raw(f[:, :, None])[:, :, 0]
    s = np.arange(nu) - (nu - 1) / 2
    R = geo.vial_radius
    for k, th in enumerate(ang):
        s0 = cx * math.cos(th) + cy * math.sin(th)
        a = np.sqrt(np.maximum(r * r - (s - s0) ** 2, 0))
        if attenuated:
            t0 = -cx * math.sin(th) + cy * math.cos(th)
            ana = (np.exp(-mu * np.sqrt(np.maximum(R * R - s * s, 0))) * math.exp(-mu * t0)
                   * 2 * np.sinh(mu * a) / mu)
        else:
            ana = 2 * a
        err = np.linalg.norm(p[k] - ana) / np.linalg.norm(ana)
        assert err < bound, (k, err)


def test_sphere_chords_slice_separable():
    """3-D: P of a supersampled sphere vs chords 2 sqrt(R^2 - (s-s0)^2 - (z-z0)^2)."""
    n, nz, R = 48, 40, 14.0
    ss = 4
    c = np.arange(n) - (n - 1) / 2
    cz = np.arange(nz) - (nz - 1) / 2
    off = (np.arange(ss) + 0.5) / ss - 0.5
    cx, cy, c0 = 3.2, -2.1, 1.7
    f = np.zeros((n, n, nz))
    for a in off:
        for b in off:
            for e in off:
                Y, X, Z = np.meshgrid(c + a, c + b, cz + e, indexing="ij")
                f += ((X - cx) ** 2 + (Y - cy) ** 2 + (Z - c0) ** 2 <= R * R)
    f /= ss ** 3
    ang = np.array([0.3, 1.1, 2.0, 2.9])
    nu = 70
    geo = Geometry(n, n, nz, ang, nu)
    p = Operators(geo).project_raw(f)
    s = np.arange(nu) - (nu - 1) / 2
    for k, th in enumerate(ang):
        s0 = cx * math.cos(th) + cy * math.sin(th)
        ana = 2 * np.sqrt(np.maximum(R * R - (s[:, None] - s0) ** 2 - (cz[None, :] - c0) ** 2, 0))
        err = np.linalg.norm(p[k] - ana) / np.linalg.norm(ana)
        assert err < 0.05, (k, err)


def test_vial_excludes_outside_voxels_and_missed_rays():
    geo = Geometry(32, 32, 1, np.array([0.2, 1.3]), 45, vial_radius=10.0, mu=0.0)
    PT = backprojector_matrix(geo)
    xs = np.arange(32) - 15.5
    Y, X = np.meshgrid(xs, xs, indexing="ij")
    outside = (X * X + Y * Y > 100.0).ravel()
    assert PT[outside].nnz == 0
    # rays whose bin centre misses the vial carry nothing
    s = np.arange(45) - 22.0
    miss = np.tile(np.abs(s) > 10.0, 2)
    assert PT[:, miss].nnz == 0


def test_adjointness_with_psf_and_attenuation():
    rng = np.random.default_rng(3)
    geo = Geometry(18, 18, 9, rng.uniform(0, np.pi, 7), 27, vial_radius=8.5, mu=0.03,
                   psf_sigma=(1.0, 0.7, 1.3))
    ops = Operators(geo)
    p = rng.normal(size=geo.vol_shape)
    y = rng.normal(size=geo.sino_shape)
    lhs = np.sum(ops.A(p) * y)
    rhs = np.sum(p * ops.AT(y))
    assert abs(lhs - rhs) <= 1e-12 * np.linalg.norm(p) * np.linalg.norm(y) * 50


def test_psf_impulse_taps_and_library_convolution():
    sig = (1.5, 1.0, 2.5)
    geo = Geometry(16, 16, 16, np.zeros(1), 16, psf_sigma=sig)
    R = geo.psf_radii()
    assert R == (6, 4, 10)
    kx, ky, kz = (psf_taps(s, r) for s, r in zip(sig, R))
    for k in (kx, ky, kz):
        assert abs(k.sum() - 1) < 1e-15
        np.testing.assert_allclose(k, k[::-1])
    imp = np.zeros((16, 16, 16))
    imp[8, 7, 8] = 1.0
    out = apply_psf(geo, imp)
    kern = ky[:, None, None] * kx[None, :, None] * kz[None, None, :]
    # impulse response: the separable kernel, clipped to the grid
    np.testing.assert_allclose(out[8 - 4:8 + 5, 7 - 6:7 + 7, :],
                               kern[:, :, 10 - 8:10 + 8], rtol=1e-13, atol=1e-17)
    rng = np.random.default_rng(4)
    a = rng.normal(size=(16, 16, 16))
    ref = ndimage.convolve(a, kern, mode="constant", cval=0.0)
    np.testing.assert_allclose(apply_psf(geo, a), ref, rtol=1e-11, atol=1e-13)
    b = rng.normal(size=(16, 16, 16))
    assert abs(np.sum(apply_psf(geo, a) * b) - np.sum(a * apply_psf(geo, b))) < 1e-11


def test_paper_psf_is_radius_two_unit_gaussian():
    """Sec. 3.4: a 21^3 kernel whose central 5^3 holds a sigma=1 Gaussian == radius 2."""
    geo = Geometry(8, 8, 8, np.zeros(1), 8, psf_sigma=(1.0, 1.0, 1.0), psf_trunc=2.0)
    assert geo.psf_radii() == (2, 2, 2)
    k = psf_taps(1.0, 2)
    e = np.exp(-np.array([4, 1, 0, 1, 4]) / 2.0)
    np.testing.assert_allclose(k, e / e.sum(), rtol=1e-15)


@pytest.mark.parametrize("axis", [0, 1, 2])
def test_psf_sigma_gradient_matches_finite_differences(axis):
    rng = np.random.default_rng(5 + axis)
    sig = [1.5, 1.2, 2.0]
    geo = Geometry(24, 24, 24, np.zeros(1), 24, psf_sigma=tuple(sig))
    R = geo.psf_radii()
    a = rng.normal(size=geo.vol_shape)
    b = rng.normal(size=geo.vol_shape)
    grad = np.sum(b * apply_psf(geo, a, deriv_axis=axis))
    h = 1e-4
    sp_, sm_ = list(sig), list(sig)
    sp_[axis] += h
    sm_[axis] -= h
    fd = (np.sum(b * apply_psf(geo, a, sigma=sp_, radii=R))
          - np.sum(b * apply_psf(geo, a, sigma=sm_, radii=R))) / (2 * h)
    assert abs(grad - fd) <= 1e-6 * abs(grad)
    # the derivative taps integrate to zero (the taps stay normalised)
    assert abs(psf_tap_derivative(sig[axis], R[axis]).sum()) < 1e-15


def test_f32_detector_coordinate_is_fused_multiply_add():
    """The 'f32' emulation equals round32(x*c + round32(y*s + off)) in exact rationals."""
    rng = np.random.default_rng(6)

    def r32(q):
        return Fraction(float(np.float32(float(q))))   # float(q) exact enough? check below

    for _ in range(200):
        n = int(rng.integers(8, 600))
        x = int(rng.integers(0, n)) - (n - 1) / 2
        y = int(rng.integers(0, n)) - (n - 1) / 2
        th = rng.uniform(0, 2 * np.pi)
        off = (int(rng.integers(8, 800)) - 1) / 2
        c32 = Fraction(float(np.float32(math.cos(th))))
        s32 = Fraction(float(np.float32(math.sin(th))))
        o32 = Fraction(float(np.float32(off)))
        inner_exact = Fraction(y) * s32 + o32
        # float(Fraction) rounds correctly to double; the exact value has < 53
        # significant bits here, so the double is exact and np.float32 rounds once
        assert Fraction(float(inner_exact)) == inner_exact
        inner = r32(inner_exact)
        outer_exact = Fraction(x) * c32 + inner
        assert Fraction(float(outer_exact)) == outer_exact
        u = r32(outer_exact)
        got = detector_coordinate(np.float64(x), np.float64(y), math.cos(th), math.sin(th),
                                  off, "f32")
        assert Fraction(float(got)) == u


def test_single_output_samplers_agree_with_matrices():
    rng = np.random.default_rng(7)
    geo = Geometry(20, 20, 6, rng.uniform(0, np.pi, 9), 29, vial_radius=9.0, mu=0.02,
                   psf_sigma=(1.0, 1.5, 0.8))
    ops = Operators(geo)
    vol = rng.uniform(size=geo.vol_shape)
    sino = rng.uniform(size=geo.sino_shape)
    bp = ops.backproject_raw(sino)
    pr = ops.project_raw(vol)
    kv = apply_psf(geo, vol)
    for _ in range(20):
        iy, ix, iz = rng.integers(0, 20), rng.integers(0, 20), rng.integers(0, 6)
        assert abs(sample.backproject_voxel(geo, sino, iy, ix, iz) - bp[iy, ix, iz]) < 1e-12
        assert abs(sample.psf_voxel(geo, vol, iy, ix, iz) - kv[iy, ix, iz]) < 1e-12
        k, j = rng.integers(0, 9), rng.integers(0, 29)
        assert abs(sample.project_ray(geo, vol, k, j, iz) - pr[k, j, iz]) < 1e-12


@pytest.mark.parametrize("n, n_angles, n_det", [(64, 96, 91), (64, 360, 64), (48, 180, 67)])
def test_active_set_readings_differ_only_on_grazing_rays(n, n_angles, n_det):
    """Sec. 2.2 defines the active rays as {[P f_T]_j > 0}.  The FP32 kernels
    decide it with their own u (two fused multiply-adds in single precision),
    the FP64 definition with u in double.  With f_T >= 0 and weights
    max(0, 1 - |u - j|), a ray can change sides only through a tap whose
    weight is within single-precision rounding of zero (u within ~1e-5 of
    j -+ 1), so every ray on which the two readings differ carries an FP64
    value of at most a few such weights; the test bounds that value and
    reports how many rays differ."""
    tgt = discs_2d(n, n_discs=3, r_range=(n / 10, n / 5), container_radius=n / 2 - 4, seed=4)
    geo = Geometry(n, n, 1, uniform_angles(n_angles), n_det)
    v64 = backprojector_matrix(geo, precision="f64").T @ tgt.ravel().astype(np.float64)
    v32 = backprojector_matrix(geo, precision="f32").T @ tgt.ravel().astype(np.float64)
    diff = (v64 > 0) != (v32 > 0)
    print(f"active rays: {int((v64 > 0).sum())} (FP64), {int((v32 > 0).sum())} (FP32 u), "
          f"{int(diff.sum())} differ of {diff.size}")
    assert diff.sum() <= 1e-2 * diff.size
    assert np.all(v64[diff] <= 4 * 2.0 ** -16 * n) and np.all(v32[diff] <= 4 * 2.0 ** -16 * n)
