"""Post-solve metrics of the GPU solve against the oracle (GPU).

After a solve the library reports DTVR_f and DSR (Eqs. 6-8), PSR_f (Eq. 46),
the post-scaling factor alpha* (Eq. 27) and the recovered Charnes-Cooper
scale s.  Each test compares them with `oracle.lp.metrics` twice: on the
dose field the GPU returns (same input, so only the reductions differ:
<= 1e-12), and on the dose the oracle recomputes in FP64 from the GPU's own
y (so the operator's rounding enters too: <= 1e-10 for FP64 solves, <= 1e-5
for FP32).
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle.lp import CaseParams, build_lp, metrics
from oracle.operators import Geometry
from synthetic.targets import csg_3d, discs_2d, graded_discs_2d, uniform_angles

KEYS = ("dtvr_f", "dsr", "psr_f", "alpha", "s")


@pytest.fixture(scope="module")
def sipo():
    import paper_2604_08997_gb300 as s
    s.build()
    return s


def _compare(sipo, ctx, res, lp, ops, geo, dtype, op_tol):
    np_dt = np.float64 if dtype == "f64" else np.float32
    d = np.empty(geo.vol_shape, np_dt)
    y = np.empty(geo.sino_shape, np_dt)
    sipo.sipo_get_array(ctx, 5, d)
    sipo.sipo_get_array(ctx, 2, y)
    same = metrics(lp, d.astype(np.float64))
    fresh = metrics(lp, ops.AT(y.astype(np.float64)).ravel())
    for k in KEYS:
        # s divides by the LP's normalised profile f~ = f_T / f_crit, which an
        # FP32 context holds in FP32 (one rounding, relative <= 2^-24); the other
        # metrics use f_T and f_crit as given
        rel = 2.4e-7 if (k == "s" and dtype == "f32") else 1e-12
        assert res[k] == pytest.approx(same[k], rel=rel, abs=1e-300), (k, res[k], same[k])
        assert res[k] == pytest.approx(fresh[k], rel=op_tol), (k, res[k], fresh[k])


TINY = [(0, {}), (1, dict(tol_lo=0.1, tol_hi=0.1)), (2, dict(inhibit_ratio=0.6))]


@pytest.mark.parametrize("case,extra", TINY)
def test_tiny_fp64_metrics_match_the_oracle(sipo, case, extra):
    n, na, nd = 10, 8, 15
    tgt = discs_2d(n, n_discs=1, r_range=(2.0, 3.0), container_radius=4.0, seed=3)
    ang = uniform_angles(na)
    g = Geometry(n, n, 1, ang, nd)
    lp, ops = build_lp(g, tgt, CaseParams(case=case, band_width=2, **extra))
    ctx = sipo.sipo_create(dict(nx=n, ny=n, nz=1, angles=ang, n_det=nd), tgt,
                           dict(kase=case, band_width=2, **extra),
                           dict(storage=sipo.SIPO_F64, kkt_tol=1e-9, max_iter=100000))
    res = sipo.sipo_solve(ctx)
    assert res["status"] == sipo.SIPO_OPTIMAL
    _compare(sipo, ctx, res, lp, ops, g, "f64", 1e-10)
    sipo.sipo_destroy(ctx)


@pytest.mark.parametrize("case,extra", TINY)
def test_multilevel_metrics_match_the_oracle(sipo, case, extra):
    """A multi-level target puts a per-voxel f~ into the ratios of Eqs. 6-8."""
    n, na, nd = 12, 10, 17
    tgt = graded_discs_2d(n, levels=(1.0, 0.6, 0.8), r_range=(1.5, 3.0), container_radius=4.5, seed=4)
    ang = uniform_angles(na)
    g = Geometry(n, n, 1, ang, nd)
    lp, ops = build_lp(g, tgt, CaseParams(case=case, band_width=2, **extra))
    for storage, dt, op_tol in ((sipo.SIPO_F64, "f64", 1e-10), (sipo.SIPO_F32, "f32", 1e-5)):
        ctx = sipo.sipo_create(dict(nx=n, ny=n, nz=1, angles=ang, n_det=nd), tgt,
                               dict(kase=case, band_width=2, **extra),
                               dict(storage=storage, kkt_tol=0.0, max_iter=512))
        res = sipo.sipo_solve(ctx)
        _compare(sipo, ctx, res, lp, ops, g, dt, op_tol)
        sipo.sipo_destroy(ctx)


@pytest.mark.parametrize("case,extra", [(1, dict(tol_lo=0.05, tol_hi=0.05)), (2, dict(inhibit_ratio=0.8))])
def test_csg48_fp32_metrics_match_the_oracle(sipo, case, extra):
    """A 3-D CSG part (48^3, 68 views, vial) after 1024 FP32 iterations: the
    metrics pass runs on the full volume with z in the vector lanes."""
    n = 48
    tgt = csg_3d(n, vial_radius=22.5, band_width=2, seed=2, feature=(3.0, 12.0))
    ang = uniform_angles(68)
    g = Geometry(n, n, n, ang, n, vial_radius=22.5)
    lp, ops = build_lp(g, tgt, CaseParams(case=case, band_width=2, **extra))
    ctx = sipo.sipo_create(dict(nx=n, ny=n, nz=n, angles=ang, n_det=n, vial_radius=22.5), tgt,
                           dict(kase=case, band_width=2, **extra),
                           dict(storage=sipo.SIPO_F32, kkt_tol=0.0, max_iter=1024))
    res = sipo.sipo_solve(ctx)
    _compare(sipo, ctx, res, lp, ops, g, "f32", 1e-5)
    sipo.sipo_destroy(ctx)
