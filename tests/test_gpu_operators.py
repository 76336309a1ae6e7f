"""GPU parity of the operators, setup arrays and autograd against the CPU oracle.

Every comparison goes through the C ABI.  Tolerances: FP32 relative L2 <= 1e-5
(the bound the projector is held to); FP64 relative L2 <= 1e-12 (rounding of
~1e3-term sums of O(1) values).  Integer outputs (labels, active-ray mask) must
match bit for bit, with the mask decided in the kernel's precision.
"""
import math

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle import sample
from oracle.lp import partition
from oracle.operators import Geometry, Operators, apply_psf, backprojector_matrix
from synthetic.targets import csg_3d, uniform_angles

FP32_TOL = 1e-5
FP64_TOL = 1e-12


@pytest.fixture(scope="module")
def sipo():
    import paper_2604_08997_gb300 as s
    s.build()
    return s


def _rel(a, b):
    return float(np.linalg.norm(np.asarray(a, np.float64) - b) / max(np.linalg.norm(b), 1e-300))


CASES = [
    # (nx, ny, nz, n_angles, n_det, vial, mu, sigma): ragged sizes, scalar and vector z paths
    (37, 29, 13, 23, 51, 0.0, 0.0, (0.0, 0.0, 0.0)),
    (24, 24, 16, 19, 35, 11.0, 0.03, (0.0, 0.0, 0.0)),
    (21, 26, 24, 31, 37, 10.5, 0.02, (1.0, 0.7, 1.3)),
    (33, 33, 1, 45, 47, 0.0, 0.0, (0.0, 0.0, 0.0)),
    # deep z: two 16-byte groups per lane (FP32 at nz % 256 == 0, FP64 at nz % 128 == 0)
    (11, 9, 256, 7, 15, 4.0, 0.05, (0.0, 0.0, 0.0)),
    # one group per lane with a partly idle last warp (132 = 128 + 4)
    (10, 12, 132, 9, 17, 0.0, 0.0, (0.0, 0.0, 0.0)),
    # degenerate sizes: one view and one detector bin; two views, three bins, a PSF
    # wider than the grid along x
    (9, 7, 5, 1, 1, 0.0, 0.0, (0.0, 0.0, 0.0)),
    (6, 5, 8, 2, 3, 2.5, 0.1, (0.6, 0.0, 0.0)),
]


def _ctx(sipo, case, storage, seed=0, tile=-1):
    nx, ny, nz, na, nd, vial, mu, sig = case
    rng = np.random.default_rng(seed)
    ang = np.sort(rng.uniform(0, 2 * np.pi, na))
    tgt = np.zeros((ny, nx, nz), np.float32)
    tgt[ny // 3: 2 * ny // 3, nx // 3: 2 * nx // 3, nz // 4: max(nz // 4 + 1, 3 * nz // 4)] = 1.0
    geo = dict(nx=nx, ny=ny, nz=nz, angles=ang, n_det=nd, vial_radius=vial, mu=mu, psf_sigma=sig)
    ctx = sipo.sipo_create(geo, tgt, dict(kase=0, band_width=2),
                           dict(storage=storage, max_iter=0, tile_cfg=tile))
    ogeo = Geometry(nx, ny, nz, ang, nd, vial_radius=vial, mu=mu, psf_sigma=sig)
    return ctx, ogeo, tgt


@pytest.mark.parametrize("case", CASES)
@pytest.mark.parametrize("storage", ["f32", "f64"])
def test_operator_pair_matches_oracle(sipo, case, storage):
    st = sipo.SIPO_F32 if storage == "f32" else sipo.SIPO_F64
    dt = torch.float32 if storage == "f32" else torch.float64
    ctx, ogeo, _ = _ctx(sipo, case, st)
    ops = Operators(ogeo)
    rng = np.random.default_rng(1)
    vol = rng.uniform(-1, 1, size=ogeo.vol_shape)
    sino = rng.uniform(-1, 1, size=ogeo.sino_shape)
    out_s = torch.empty(ogeo.sino_shape, dtype=dt, device="cuda")
    out_v = torch.empty(ogeo.vol_shape, dtype=dt, device="cuda")
    sipo.sipo_project(ctx, torch.tensor(vol, dtype=dt, device="cuda"), out_s)
    sipo.sipo_backproject(ctx, torch.tensor(sino, dtype=dt, device="cuda"), out_v)
    torch.cuda.synchronize()
    tol = FP32_TOL if storage == "f32" else FP64_TOL
    assert _rel(out_s.cpu().numpy(), ops.A(vol)) <= tol
    assert _rel(out_v.cpu().numpy(), ops.AT(sino)) <= tol
    # adjointness of the GPU pair itself
    lhs = float(torch.sum(out_s.double() * torch.tensor(sino, device="cuda")))
    rhs = float(torch.sum(out_v.double() * torch.tensor(vol, device="cuda")))
    assert abs(lhs - rhs) <= (1e-5 if storage == "f32" else 1e-12) * math.sqrt(vol.size * sino.size)


@pytest.mark.parametrize("case", CASES)
def test_every_backprojector_tile_matches_the_oracle(sipo, case):
    """Each entry of the backprojector tile table (0-2: per-voxel row window;
    3-4: row patterns with packed multiply-adds; 5-6: the same fed by
    tensor-memory copies into shared memory, on the z = 256 case) against the
    oracle, and the entries against each other: they add the same terms in the
    same order, so the FP32 sums agree bit for bit."""
    n_tiles = sipo.sipo_tile_count()
    assert n_tiles == 7
    outs = []
    for tile in range(n_tiles):
        ctx, ogeo, _ = _ctx(sipo, case, sipo.SIPO_F32, tile=tile)
        ops = Operators(ogeo)
        rng = np.random.default_rng(7)
        sino = rng.uniform(-1, 1, size=ogeo.sino_shape)
        out_v = torch.empty(ogeo.vol_shape, dtype=torch.float32, device="cuda")
        sipo.sipo_backproject(ctx, torch.tensor(sino, dtype=torch.float32, device="cuda"), out_v)
        torch.cuda.synchronize()
        o = out_v.cpu().numpy()
        assert _rel(o, ops.AT(sino)) <= FP32_TOL, tile
        outs.append(o)
        sipo.sipo_destroy(ctx)
    for tile in range(1, n_tiles):
        np.testing.assert_array_equal(outs[tile], outs[0], err_msg=f"tile {tile}")


@pytest.mark.parametrize("storage", ["f32", "f64"])
def test_labels_and_active_mask_bit_exact(sipo, storage):
    st = sipo.SIPO_F32 if storage == "f32" else sipo.SIPO_F64
    for case in CASES:
        ctx, ogeo, tgt = _ctx(sipo, case, st, seed=2)
        lab = np.empty(ogeo.vol_shape, np.uint8)
        act = np.empty(ogeo.sino_shape, np.uint8)
        sipo.sipo_get_array(ctx, 0, lab)
        sipo.sipo_get_array(ctx, 1, act)
        np.testing.assert_array_equal(lab, partition(ogeo, tgt, 2))
        # the active set is an integer decision taken in the kernel's precision
        PT = backprojector_matrix(ogeo, precision=storage)
        nz = ogeo.nz
        pf = (PT.T @ tgt.reshape(-1, nz).astype(np.float64)).reshape(ogeo.sino_shape)
        np.testing.assert_array_equal(act, (pf > 0).astype(np.uint8))


@pytest.mark.parametrize("axis", [-1, 0, 1, 2])
def test_psf_and_sigma_derivative(sipo, axis):
    case = CASES[2]
    ctx, ogeo, _ = _ctx(sipo, case, sipo.SIPO_F64)
    rng = np.random.default_rng(3)
    vol = rng.normal(size=ogeo.vol_shape)
    out = torch.empty(ogeo.vol_shape, dtype=torch.float64, device="cuda")
    sipo.sipo_psf_apply(ctx, torch.tensor(vol, device="cuda"), out, axis)
    ref = apply_psf(ogeo, vol, deriv_axis=None if axis < 0 else axis)
    assert _rel(out.cpu().numpy(), ref) <= FP64_TOL


PSF_F32 = [
    (21, 26, 24, 31, 37, 10.5, 0.02, (1.0, 0.7, 1.3)),    # z groups ragged in the 16-value tile
    (37, 29, 132, 5, 41, 0.0, 0.0, (1.5, 1.5, 2.5)),      # radii 6, 6, 10; two z chunks, the last ragged
    (20, 18, 256, 5, 23, 0.0, 0.0, (2.0, 0.0, 3.0)),      # radii 8, 0, 12
    (19, 23, 13, 5, 25, 0.0, 0.0, (1.2, 0.9, 0.8)),       # nz % 4 != 0: the three-pass kernels
]


@pytest.mark.parametrize("case", PSF_F32)
@pytest.mark.parametrize("axis", [-1, 0, 1, 2])
def test_psf_fp32_matches_the_oracle(sipo, case, axis):
    """Single-precision K (and its sigma derivative along one axis): the fused
    x-y pass through shared memory and the chunked z pass (nz % 4 == 0), or
    the three per-axis passes, against the oracle's direct convolution.  Three
    FP32 passes of <= 25 taps each, taps rounded to FP32: relative L2 <= 2e-6
    (about 3e-7 expected per pass for sums of random-sign terms)."""
    ctx, ogeo, _ = _ctx(sipo, case, sipo.SIPO_F32)
    if axis >= 0 and ogeo.psf_sigma[axis] == 0.0:
        pytest.skip("no blur along this axis")
    rng = np.random.default_rng(4)
    vol = rng.normal(size=ogeo.vol_shape).astype(np.float32)
    out = torch.empty(ogeo.vol_shape, dtype=torch.float32, device="cuda")
    sipo.sipo_psf_apply(ctx, torch.tensor(vol, device="cuda"), out, axis)
    torch.cuda.synchronize()
    ref = apply_psf(ogeo, vol.astype(np.float64), deriv_axis=None if axis < 0 else axis)
    assert _rel(out.cpu().numpy(), ref) <= 2e-6


@pytest.mark.parametrize("n,sigma", [(256, (1.5, 1.5, 2.5)), (512, (2.0, 2.0, 3.0))])
def test_full_size_psf_sampled(sipo, n, sigma):
    """K at the sizes of the blurred workloads (256^3 with sigma (1.5, 1.5,
    2.5), 512^3 with (2, 2, 3)), in the launch configuration the solver uses
    (fused x-y pass, chunked z pass): sampled outputs, grid edges and corners
    included, against the oracle's direct box sum one by one."""
    geo = dict(nx=n, ny=n, nz=n, angles=uniform_angles(4), n_det=n, psf_sigma=sigma)
    tgt = np.zeros((n, n, n), np.float32)
    tgt[n // 3: n // 2, n // 3: n // 2, n // 3: n // 2] = 1.0
    ctx = sipo.sipo_create(geo, tgt, dict(kase=0, band_width=2),
                           dict(storage=sipo.SIPO_F32, max_iter=0, tile_cfg=4))
    ogeo = Geometry(n, n, n, uniform_angles(4), n, psf_sigma=sigma)
    g = torch.Generator(device="cuda").manual_seed(8)
    vol = torch.rand((n, n, n), device="cuda", generator=g)
    out = torch.empty_like(vol)
    sipo.sipo_psf_apply(ctx, vol, out, -1)
    torch.cuda.synchronize()
    rng = np.random.default_rng(9)
    pts = [(0, 0, 0), (n - 1, n - 1, n - 1), (0, n - 1, 5), (n // 2, 0, n - 1)]
    pts += [tuple(int(v) for v in rng.integers(0, n, 3)) for _ in range(20)]
    vol_h = None
    errs = []
    for iy, ix, iz in pts:
        if vol_h is None:
            vol_h = vol.cpu().numpy()
        ref = sample.psf_voxel(ogeo, vol_h, iy, ix, iz)
        errs.append(abs(float(out[iy, ix, iz]) - ref) / max(abs(ref), 1e-3))
    assert max(errs) <= 2e-6, max(errs)
    sipo.sipo_destroy(ctx)


@pytest.mark.parametrize("n,na,vial,mu", [(256, 360, 120.0, 0.005), (512, 720, 240.0, 0.0025)])
def test_full_size_sampled_outputs(sipo, n, na, vial, mu):
    """256^3 x 360 views (the solver's measured configuration, with
    attenuation) and 512^3 x 720 views (the large part's geometry): sampled
    outputs of the same launch configuration checked one by one against the
    oracle, and the adjointness of the whole launch."""
    ang = uniform_angles(na)
    geo = dict(nx=n, ny=n, nz=n, angles=ang, n_det=n, vial_radius=vial, mu=mu)
    tgt = csg_3d(n, vial_radius=vial, band_width=10, seed=2)
    ctx = sipo.sipo_create(geo, tgt, dict(kase=2, band_width=10, inhibit_ratio=0.8),
                           dict(storage=sipo.SIPO_F32, max_iter=0))
    ogeo = Geometry(n, n, n, ang, n, vial_radius=vial, mu=mu)
    g = torch.Generator(device="cuda").manual_seed(5)
    vol = torch.rand((n, n, n), device="cuda", generator=g)
    sino = torch.rand((na, n, n), device="cuda", generator=g)
    out_s = torch.empty_like(sino)
    out_v = torch.empty_like(vol)
    sipo.sipo_project(ctx, vol, out_s)
    sipo.sipo_backproject(ctx, sino, out_v)
    torch.cuda.synchronize()
    vol_h, sino_h = vol.cpu().numpy(), sino.cpu().numpy()
    s_h, v_h = out_s.cpu().numpy(), out_v.cpu().numpy()
    rng = np.random.default_rng(6)
    errs_v, errs_s = [], []
    for _ in range(24):
        iy, ix, iz = (int(v) for v in rng.integers(0, n, 3))
        ref = sample.backproject_voxel(ogeo, sino_h, iy, ix, iz)
        errs_v.append(abs(v_h[iy, ix, iz] - ref) / max(abs(ref), 1.0))
        k, j, iz = int(rng.integers(0, na)), int(rng.integers(0, n)), int(rng.integers(0, n))
        ref = sample.project_ray(ogeo, vol_h, k, j, iz)
        errs_s.append(abs(s_h[k, j, iz] - ref) / max(abs(ref), 1.0))
    assert max(errs_v) <= 1e-5 and max(errs_s) <= 1e-5, (max(errs_v), max(errs_s))
    # property at full size: adjointness of the whole launch
    lhs = float(torch.sum(out_s.double() * sino.double()))
    rhs = float(torch.sum(out_v.double() * vol.double()))
    assert abs(lhs - rhs) <= 1e-5 * abs(lhs)
    sipo.sipo_destroy(ctx)


def test_autograd_gradcheck_and_sigma_fd(sipo):
    from paper_2604_08997_gb300 import autograd as ag
    case = (10, 9, 8, 7, 15, 4.5, 0.05, (0.9, 0.7, 1.1))
    ctx, ogeo, _ = _ctx(sipo, case, sipo.SIPO_F64)
    p = torch.rand(ogeo.vol_shape, dtype=torch.float64, device="cuda", requires_grad=True)
    y = torch.rand(ogeo.sino_shape, dtype=torch.float64, device="cuda", requires_grad=True)
    sig = torch.tensor([0.9, 0.7, 1.1], dtype=torch.float64, requires_grad=True)
    assert torch.autograd.gradcheck(lambda a, s: ag.project(ctx, a, s), (p, sig), eps=1e-6,
                                    atol=1e-7, rtol=1e-6)
    assert torch.autograd.gradcheck(lambda a, s: ag.backproject(ctx, a, s), (y, sig), eps=1e-6,
                                    atol=1e-7, rtol=1e-6)
    # sigma gradient of <w, A p> against central differences with the radius frozen
    w = torch.rand(ogeo.sino_shape, dtype=torch.float64, device="cuda")
    loss = torch.sum(w * ag.project(ctx, p.detach(), sig))
    (gs,) = torch.autograd.grad(loss, sig)
    h = 1e-4
    for a in range(3):
        sp, sm = sig.detach().clone(), sig.detach().clone()
        sp[a] += h
        sm[a] -= h
        fp = float(torch.sum(w * ag.project(ctx, p.detach(), sp)))
        fm = float(torch.sum(w * ag.project(ctx, p.detach(), sm)))
        fd = (fp - fm) / (2 * h)
        assert abs(float(gs[a]) - fd) <= 1e-6 * max(1.0, abs(fd))
    sipo.sipo_set_psf_sigma(ctx, [0.9, 0.7, 1.1])
