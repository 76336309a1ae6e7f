"""Full-size certificate: the 256^3 x 360-view solve re-evaluated by the oracle (GPU).

The measured workload (256^3 voxels, 360 views over [0, pi), 256 x 256
detector, vial of radius 120, Case 2) is solved in FP32 at the inhibition
ratio 0.85, where it converges to a relative KKT error of 1e-4.  The
returned primal-dual point (y, lam_up, lam_lo, u~, v~) is then re-evaluated by
the FP64 oracle: A^T y and A (lam_up - lam_lo) with the oracle's explicit
operator, the residuals, objectives and relative KKT error of Sec. 6.1.  The
point is a certificate of near-optimality only if the FP64 evaluation agrees;
FP32 storage of y and the duals, and the FP32 operator, allow twice the
solver's tolerance.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle.lp import CaseParams, build_lp, kkt
from oracle.operators import Geometry
from synthetic.targets import workload


@pytest.fixture(scope="module")
def sipo():
    import paper_2604_08997_gb300 as s
    s.build()
    return s


def test_csg256_fp32_solve_is_an_fp64_certificate(sipo):
    wl = workload("csg256")
    n, ratio = wl.n, 0.85
    geo = dict(nx=n, ny=n, nz=wl.nz, angles=wl.angles, n_det=wl.n_det, vial_radius=wl.vial_radius)
    cp = dict(kase=2, inhibit_ratio=ratio, band_width=wl.band_width)
    ctx = sipo.sipo_create(geo, torch.from_numpy(wl.target).cuda(), cp,
                           dict(storage=sipo.SIPO_F32, kkt_tol=1e-4, max_iter=4096))
    res = sipo.sipo_solve(ctx)
    assert res["status"] == sipo.SIPO_OPTIMAL, res
    assert res["kkt"] <= 1e-4
    y = np.empty((wl.n_angles, wl.n_det, wl.nz), np.float32)
    lu = np.empty((n, n, wl.nz), np.float32)
    ll = np.empty((n, n, wl.nz), np.float32)
    sc = sipo.sipo_get_state(ctx, y, lu, ll)
    sipo.sipo_destroy(ctx)
    g3 = Geometry(n, n, wl.nz, wl.angles, wl.n_det, vial_radius=wl.vial_radius)
    lp, ops = build_lp(g3, wl.target, CaseParams(case=2, inhibit_ratio=ratio, band_width=wl.band_width))
    d = ops.AT(y.astype(np.float64)).ravel()
    g = ops.A(lu.astype(np.float64) - ll.astype(np.float64)).ravel()
    info = kkt(lp, d, g, sc["u"], sc["v"], lu, ll)
    assert info["kkt"] <= 2e-4, info
    # the primal objective is v~ itself; the dual objective is re-summed in FP64
    assert info["pobj"] == pytest.approx(res["pobj"], rel=1e-12)
    assert info["dobj"] == pytest.approx(res["dobj"], rel=1e-4)
    assert info["rel_primal"] <= 2e-4 and info["rel_dual"] <= 2e-4 and info["rel_gap"] <= 2e-4


def test_csg256_ratio_08_gpu_certificate_holds_in_fp64(sipo):
    """The headline status checked on the GPU's own certificate: the
    separation LP of the measured part (Case 1 with tol_lo = 0, tol_hi = 10)
    is solved in FP32 with Farkas probes of Case 2 at r = 0.8 until a probe
    passes on some slice z; the dual point that passed (the separation
    context's exported state) is then re-tested by the oracle in FP64 on that
    slice alone, with the slice's rows of the 3-D LP (labels of the 3-D part)
    and the bound-based test of Sec. 2.7 - one slice that cannot be met makes
    the whole slice-separable LP infeasible."""
    from oracle import pdhg
    from oracle.lp import partition
    wl = workload("csg256")
    n, r = wl.n, 0.8
    geo = dict(nx=n, ny=n, nz=wl.nz, angles=wl.angles, n_det=wl.n_det, vial_radius=wl.vial_radius)
    tgt = torch.from_numpy(wl.target).cuda()
    sep = sipo.sipo_create(geo, tgt, dict(kase=1, tol_lo=0.0, tol_hi=10.0, band_width=wl.band_width),
                           dict(storage=sipo.SIPO_F32, kkt_tol=1e-4, max_iter=16384))
    c2 = sipo.sipo_create(geo, tgt, dict(kase=2, inhibit_ratio=r, band_width=wl.band_width),
                          dict(storage=sipo.SIPO_F32, kkt_tol=1e-4, max_iter=64))
    res, certified, z = sipo.sipo_solve_probe(sep, c2, 128)
    assert certified and 0 <= z < wl.nz, (res["status_name"], certified, z)
    assert res["status"] == sipo.SIPO_ITER_LIMIT
    lu = torch.empty((n, n, wl.nz), dtype=torch.float32, device="cuda")
    ll = torch.empty_like(lu)
    y = torch.empty((wl.n_angles, wl.n_det, wl.nz), dtype=torch.float32, device="cuda")
    sipo.sipo_get_state(sep, y, lu, ll)
    # the exported point is the tested one: the library certifies it again
    again, z2 = sipo.sipo_farkas_from(c2, sep)
    assert again and z2 == z
    lab3 = partition(Geometry(n, n, n, wl.angles, n, vial_radius=wl.vial_radius), wl.target, wl.band_width)
    g2 = Geometry(n, n, 1, wl.angles, n, vial_radius=wl.vial_radius)
    lp2, ops2 = build_lp(g2, np.ascontiguousarray(wl.target[:, :, z:z + 1]),
                         CaseParams(case=2, inhibit_ratio=r, band_width=wl.band_width))
    lp2.labels = lab3[:, :, z].ravel().astype(np.uint8)
    lam_up = lu[:, :, z].double().cpu().numpy().ravel()
    lam_lo = ll[:, :, z].double().cpu().numpy().ravel()
    assert pdhg.certificate(lp2, ops2, lam_up, lam_lo, *pdhg.certificate_data(lp2, ops2))
    sipo.sipo_destroy(sep)
    sipo.sipo_destroy(c2)
