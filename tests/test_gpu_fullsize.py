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
