"""GPU PDHG solves against exact optima, the oracle PDHG and FP64 certificates.

y* is not unique (A has a large null space), so parity is on objectives, KKT
errors, feasibility and statuses, never on y element by element.  The FP64
GPU solver and the oracle implement the same restarted Halpern PDHG, so on
the same instance their iterates agree to rounding for as long as no restart
decision flips; the iteration-matched test checks that.
"""
import json
import os

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle import pdhg, simplex
from oracle.lp import CaseParams, build_lp, kkt, metrics
from oracle.operators import Geometry
from synthetic.targets import csg_3d, discs_2d, graded_discs_2d, uniform_angles, workload

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")

TINY = [(0, {}), (1, dict(tol_lo=0.1, tol_hi=0.1)), (2, dict(inhibit_ratio=0.6))]


@pytest.fixture(scope="module")
def sipo():
    import paper_2604_08997_gb300 as s
    s.build()
    return s


def _tiny(case, extra, n=10, na=8, nd=15):
    tgt = discs_2d(n, n_discs=1, r_range=(2.0, 3.0), container_radius=4.0, seed=3)
    ang = uniform_angles(na)
    lp, ops = build_lp(Geometry(n, n, 1, ang, nd), tgt, CaseParams(case=case, band_width=2, **extra))
    geo = dict(nx=n, ny=n, nz=1, angles=ang, n_det=nd)
    cp = dict(kase=case, band_width=2, **extra)
    return lp, ops, geo, tgt, cp


@pytest.mark.parametrize("case,extra", TINY)
def test_tiny_lp_fp64_matches_simplex(sipo, case, extra):
    lp, ops, geo, tgt, cp = _tiny(case, extra)
    st, obj, _ = simplex.solve_dense(lp, ops)
    ctx = sipo.sipo_create(geo, tgt, cp, dict(storage=sipo.SIPO_F64, kkt_tol=1e-10, max_iter=100000))
    res = sipo.sipo_solve(ctx)
    assert st == "optimal" and res["status"] == sipo.SIPO_OPTIMAL
    assert abs(res["pobj"] - obj) <= 1e-7 * abs(obj)
    assert abs(res["s"] - 1.0) < 1e-6          # recovered Charnes-Cooper scale t = 1/s = 1


@pytest.mark.parametrize("case,extra", TINY)
def test_tiny_lp_fp32_matches_simplex(sipo, case, extra):
    lp, ops, geo, tgt, cp = _tiny(case, extra)
    st, obj, _ = simplex.solve_dense(lp, ops)
    ctx = sipo.sipo_create(geo, tgt, cp, dict(storage=sipo.SIPO_F32, kkt_tol=1e-5, max_iter=100000))
    res = sipo.sipo_solve(ctx)
    assert res["status"] == sipo.SIPO_OPTIMAL
    assert abs(res["pobj"] - obj) <= 1e-4 * abs(obj)


def test_infeasible_case2_is_reported(sipo):
    lp, ops, geo, tgt, cp = _tiny(2, dict(inhibit_ratio=0.3))
    assert simplex.solve_dense(lp, ops)[0] == "infeasible"
    for storage in (sipo.SIPO_F64, sipo.SIPO_F32):
        ctx = sipo.sipo_create(geo, tgt, cp, dict(storage=storage, kkt_tol=1e-9, max_iter=20000))
        res = sipo.sipo_solve(ctx)
        assert res["status"] == sipo.SIPO_PRIMAL_INFEASIBLE, res


@pytest.mark.parametrize("case,extra", [(1, dict(tol_lo=0.05, tol_hi=0.05)), (2, dict(inhibit_ratio=0.7))])
def test_fp64_iterates_track_the_oracle(sipo, case, extra):
    """Same algorithm, same instance, FP64 on both sides: after 640 iterations the
    objectives, KKT errors and restart counts agree."""
    tgt = discs_2d(24, n_discs=2, r_range=(3.0, 5.0), container_radius=10.0, seed=11)
    ang = uniform_angles(32)
    lp, ops = build_lp(Geometry(24, 24, 1, ang, 35), tgt, CaseParams(case=case, band_width=3, **extra))
    ref = pdhg.solve(lp, ops, kkt_tol=0.0, max_iter=640)
    ctx = sipo.sipo_create(dict(nx=24, ny=24, nz=1, angles=ang, n_det=35), tgt,
                           dict(kase=case, band_width=3, **extra),
                           dict(storage=sipo.SIPO_F64, kkt_tol=0.0, max_iter=640))
    res = sipo.sipo_solve(ctx)
    assert res["status"] == sipo.SIPO_ITER_LIMIT and res["iters"] == 640
    assert res["restarts"] == ref["restarts"]
    for key, rkey in (("pobj", "pobj"), ("dobj", "dobj"), ("rel_primal", "rel_primal"),
                      ("rel_dual", "rel_dual")):
        a, b = res[key], ref["info"][rkey]
        assert abs(a - b) <= 1e-7 * max(abs(b), 1e-3), (key, a, b)


def _layered_target(n, nz, graded=False):
    """Per-slice disc targets that change along z, so a mix-up of z values
    between lanes or 16-byte groups changes the result; `graded` gives each
    slice's discs their own levels (a multi-level target, Sec. 3.3)."""
    t = np.empty((n, n, nz), np.float32)
    for z in range(nz):
        if graded:
            lv = (1.0, 0.85, 0.7) if z % 2 else (0.8, 1.0)
            t[:, :, z] = graded_discs_2d(n, levels=lv, r_range=(1.5, 3.0), container_radius=4.0,
                                         seed=z % 7)[:, :, 0]
        else:
            t[:, :, z] = discs_2d(n, n_discs=1, r_range=(1.5, 3.0), container_radius=4.0, seed=z % 7)[:, :, 0]
    return t


@pytest.mark.parametrize("storage,nz,iters,rtol,atol,graded,ratio",
                         [("f64", 128, 320, 1e-7, 1e-10, False, 0.6),
                          ("f32", 256, 64, 1e-4, 1e-5, False, 0.6),
                          ("f64", 128, 320, 1e-7, 1e-10, True, 0.8)])
def test_deep_z_solve_tracks_the_oracle(sipo, storage, nz, iters, rtol, atol, graded, ratio):
    """The fused solver kernels with two 16-byte groups per lane (FP64 at
    nz = 128, FP32 at nz = 256) against the FP64 oracle PDHG.  FP32 iterates
    differ from FP64 ones by rounding (~1e-7 relative per step), so the FP32
    case runs one check period and allows 1e-4 relative plus 1e-5 absolute on
    the (already normalised) residuals.  The multi-level stack runs at ratio
    0.8: at 0.6 every one of its slices is infeasible (HiGHS), which the
    slice-by-slice certificate proves at the first check."""
    n, na, nd = 10, 8, 15
    tgt = _layered_target(n, nz, graded)
    ang = uniform_angles(na)
    cp = dict(kase=2, inhibit_ratio=ratio, band_width=2)
    lp, ops = build_lp(Geometry(n, n, nz, ang, nd), tgt, CaseParams(case=2, inhibit_ratio=ratio, band_width=2))
    ref = pdhg.solve(lp, ops, kkt_tol=0.0, max_iter=iters)
    assert ref["status"] == pdhg.ITER_LIMIT
    st = sipo.SIPO_F64 if storage == "f64" else sipo.SIPO_F32
    ctx = sipo.sipo_create(dict(nx=n, ny=n, nz=nz, angles=ang, n_det=nd), tgt, cp,
                           dict(storage=st, kkt_tol=0.0, max_iter=iters))
    res = sipo.sipo_solve(ctx)
    assert res["status"] == sipo.SIPO_ITER_LIMIT and res["iters"] == iters
    assert res["restarts"] == ref["restarts"]
    for key in ("pobj", "dobj", "rel_primal", "rel_dual"):
        a, b = res[key], ref["info"][key]
        assert abs(a - b) <= rtol * abs(b) + atol, (key, a, b)


GRAY = [(0, {}), (1, dict(tol_lo=0.1, tol_hi=0.1)), (2, dict(inhibit_ratio=0.9))]


@pytest.mark.parametrize("case,extra", GRAY)
def test_grayscale_target_reaches_the_oracle_optimum(sipo, case, extra):
    """A multi-level target (one level per disc, Sec. 3.3) puts a per-voxel
    normalised profile f~ into every solver kernel; the GPU solves in FP64 and
    FP32 reach the oracle PDHG's optimum (the oracle's own value is pinned to
    HiGHS on the dose-unit LP by the CPU tests)."""
    n, na, nd = 10, 8, 15
    tgt = graded_discs_2d(n, levels=(1.0, 0.85, 0.7), r_range=(1.5, 3.0), container_radius=4.0, seed=4)
    ang = uniform_angles(na)
    lp, ops = build_lp(Geometry(n, n, 1, ang, nd), tgt, CaseParams(case=case, band_width=2, **extra))
    ref = pdhg.solve(lp, ops, kkt_tol=1e-10, max_iter=80000)
    assert ref["status"] == pdhg.OPTIMAL
    geo = dict(nx=n, ny=n, nz=1, angles=ang, n_det=nd)
    cp = dict(kase=case, band_width=2, **extra)
    for storage, tol, rel in ((sipo.SIPO_F64, 1e-10, 1e-7), (sipo.SIPO_F32, 1e-5, 1e-4)):
        ctx = sipo.sipo_create(geo, tgt, cp, dict(storage=storage, kkt_tol=tol, max_iter=100000))
        res = sipo.sipo_solve(ctx)
        assert res["status"] == sipo.SIPO_OPTIMAL, (storage, res)
        assert abs(res["pobj"] - ref["obj"]) <= rel * abs(ref["obj"]), (storage, res["pobj"], ref["obj"])
        if storage == sipo.SIPO_F64:
            assert abs(res["s"] - 1.0) < 1e-6


def test_disc64_case1_fp64_to_1e6(sipo):
    """The 64x64 / 96-angle / 91-bin single-slice workload, Case 1, to KKT 1e-6."""
    wl = workload("disc64")
    ctx = sipo.sipo_create(dict(nx=64, ny=64, nz=1, angles=wl.angles, n_det=91), wl.target,
                           dict(kase=1, tol_lo=0.05, tol_hi=0.05, band_width=10),
                           dict(storage=sipo.SIPO_F64, kkt_tol=1e-6, max_iter=200000))
    res = sipo.sipo_solve(ctx)
    assert res["status"] == sipo.SIPO_OPTIMAL, res
    with open(os.path.join(GOLDEN, "disc64_case1.json")) as f:
        gold = json.load(f)
    assert abs(res["pobj"] - gold["objective"]) <= 1e-5 * gold["objective"]
    # certificate: the oracle re-evaluates the returned point in FP64
    lp, ops = build_lp(Geometry(64, 64, 1, wl.angles, 91), wl.target,
                       CaseParams(case=1, tol_lo=0.05, tol_hi=0.05, band_width=10))
    y = np.empty((96, 91, 1), np.float64)
    lu = np.empty((64, 64, 1), np.float64)
    ll = np.empty((64, 64, 1), np.float64)
    sipo.sipo_get_array(ctx, 2, y)
    sipo.sipo_get_array(ctx, 3, lu)
    sipo.sipo_get_array(ctx, 4, ll)
    d = ops.AT(y).ravel()
    g = ops.A(lu - ll).ravel()
    info = kkt(lp, d, g, res["u"], res["v"], lu, ll)
    assert info["kkt"] <= 1.01e-6
    assert abs(info["pobj"] - res["pobj"]) <= 1e-12 * res["pobj"] + 1e-15


def test_csg_case2_fp32_certificate_and_bf16(sipo):
    """A reduced 3-D CSG instance (48^3, 68 views, vial, Case 2): FP32 solve to
    1e-4, checked by an FP64 re-evaluation of its own certificate and against the
    oracle optimum; BF16 storage reports the KKT it reaches."""
    n = 48
    tgt = csg_3d(n, vial_radius=22.5, band_width=2, seed=2, feature=(3.0, 12.0))
    ang = uniform_angles(68)
    geo = dict(nx=n, ny=n, nz=n, angles=ang, n_det=n, vial_radius=22.5)
    cp = dict(kase=2, inhibit_ratio=0.8, band_width=2)
    lp, ops = build_lp(Geometry(n, n, n, ang, n, vial_radius=22.5), tgt,
                       CaseParams(case=2, inhibit_ratio=0.8, band_width=2))
    ref = pdhg.solve(lp, ops, kkt_tol=1e-5, max_iter=60000)
    ctx = sipo.sipo_create(geo, tgt, cp, dict(storage=sipo.SIPO_F32, kkt_tol=1e-4, max_iter=60000))
    res = sipo.sipo_solve(ctx)
    if ref["status"] == pdhg.PRIMAL_INFEASIBLE:
        assert res["status"] == sipo.SIPO_PRIMAL_INFEASIBLE
        return
    assert res["status"] == sipo.SIPO_OPTIMAL, res
    y = np.empty(lp.active.shape, np.float32)
    lu = np.empty(lp.labels.shape, np.float32)
    ll = np.empty(lp.labels.shape, np.float32)
    sipo.sipo_get_array(ctx, 2, y)
    sipo.sipo_get_array(ctx, 3, lu)
    sipo.sipo_get_array(ctx, 4, ll)
    g = Geometry(n, n, n, ang, n, vial_radius=22.5)
    d = ops.AT(y.reshape(g.sino_shape)).ravel()
    gg = ops.A((lu.astype(np.float64) - ll).reshape(g.vol_shape)).ravel()
    info = kkt(lp, d, gg, res["u"], res["v"], lu, ll)
    assert info["kkt"] <= 2e-4, info
    assert abs(res["pobj"] - ref["obj"]) <= 1e-3 * abs(ref["obj"])
    ctx16 = sipo.sipo_create(geo, tgt, cp, dict(storage=sipo.SIPO_BF16, kkt_tol=1e-4, max_iter=20000))
    r16 = sipo.sipo_solve(ctx16)
    assert r16["status"] in (sipo.SIPO_OPTIMAL, sipo.SIPO_ITER_LIMIT)
    # BF16 iterates stall above 1e-4; the objective of the point they reach is
    # within its own relative KKT error of the optimum (the gap part bounds
    # |p - d| and the optimum lies between them up to the residuals), plus one
    # BF16 rounding (2^-8 relative) of the stored values it is computed from
    bound = max(r16["kkt"], 2.0 ** -8)
    assert abs(r16["pobj"] - ref["obj"]) <= bound * abs(ref["obj"]), (r16["pobj"], ref["obj"], bound)


def test_batched_solve_matches_individual_solves(sipo):
    """One graph per period for the whole batch gives the same iterates as solving
    each context alone (same kernels, deterministic reductions)."""
    specs = TINY + [(2, dict(inhibit_ratio=0.3))]
    single, ctxs = [], []
    for case, extra in specs:
        lp, ops, geo, tgt, cp = _tiny(case, extra)
        tol = dict(storage=sipo.SIPO_F64, kkt_tol=1e-9, max_iter=64 * 400)
        single.append(sipo.sipo_solve(sipo.sipo_create(geo, tgt, cp, tol)))
        ctxs.append(sipo.sipo_create(geo, tgt, cp, tol))
    batched = sipo.sipo_solve_batched(ctxs)
    for a, b in zip(single, batched):
        assert a["status"] == b["status"]
        assert a["iters"] == b["iters"]
        assert a["pobj"] == b["pobj"] and a["kkt"] == b["kkt"]
    assert batched[-1]["status"] == sipo.SIPO_PRIMAL_INFEASIBLE


@pytest.mark.parametrize("storage", ["f64", "f32"])
def test_blurred_inhibition_certified_infeasible(sipo, storage):
    """Blurred, attenuated 16^3 Case-2 part at r = 0.8: the bound-based Farkas
    certificate proves infeasibility; FP64 at the oracle's iteration."""
    n = 16
    tgt = csg_3d(n, vial_radius=n * 0.47, band_width=2, seed=2, feature=(3.0, 6.0))
    ang = uniform_angles(24)
    sig = (1.5, 1.5, 2.5)
    lp, ops = build_lp(Geometry(n, n, n, ang, n, vial_radius=n * 0.47, mu=0.08, psf_sigma=sig), tgt,
                       CaseParams(case=2, inhibit_ratio=0.8, band_width=2))
    ref = pdhg.solve(lp, ops, kkt_tol=1e-4, max_iter=1024)
    assert ref["status"] == pdhg.PRIMAL_INFEASIBLE
    st = sipo.SIPO_F64 if storage == "f64" else sipo.SIPO_F32
    ctx = sipo.sipo_create(dict(nx=n, ny=n, nz=n, angles=ang, n_det=n, vial_radius=n * 0.47, mu=0.08,
                                psf_sigma=sig), tgt, dict(kase=2, inhibit_ratio=0.8, band_width=2),
                           dict(storage=st, kkt_tol=1e-4, max_iter=1024))
    res = sipo.sipo_solve(ctx)
    assert res["status"] == sipo.SIPO_PRIMAL_INFEASIBLE, res
    if storage == "f64":
        assert res["iters"] == ref["iters"]


def test_warm_start_continues_from_the_source_point(sipo):
    """A solve warm-started from a finished FP64 solve of the same problem stops
    at its first check with the same objective; a context holding another
    problem is refused."""
    case, extra = TINY[2]
    lp, ops, geo, tgt, cp = _tiny(case, extra)
    tol = dict(storage=sipo.SIPO_F64, kkt_tol=1e-9, max_iter=100000)
    src = sipo.sipo_create(geo, tgt, cp, tol)
    r0 = sipo.sipo_solve(src)
    assert r0["status"] == sipo.SIPO_OPTIMAL
    dst = sipo.sipo_create(geo, tgt, cp, tol)
    sipo.sipo_warm_start(dst, src)
    r1 = sipo.sipo_solve(dst)
    assert r1["status"] == sipo.SIPO_OPTIMAL and r1["iters"] <= 64
    assert abs(r1["pobj"] - r0["pobj"]) <= 1e-8 * abs(r0["pobj"])
    other = sipo.sipo_create(geo, tgt, dict(cp, inhibit_ratio=0.7), tol)
    with pytest.raises(sipo.SipoError):
        sipo.sipo_warm_start(other, src)


def test_bf16_escalated_to_fp32_reaches_the_target(sipo):
    """Precision escalation on the reduced 48^3 Case-2 instance: BF16 storage
    for at most 1024 iterations, then FP32 warm-started from its last check,
    to KKT 1e-4; the objective agrees with the oracle optimum."""
    n = 48
    tgt = csg_3d(n, vial_radius=22.5, band_width=2, seed=2, feature=(3.0, 12.0))
    ang = uniform_angles(68)
    geo = dict(nx=n, ny=n, nz=n, angles=ang, n_det=n, vial_radius=22.5)
    cp = dict(kase=2, inhibit_ratio=0.8, band_width=2)
    lp, ops = build_lp(Geometry(n, n, n, ang, n, vial_radius=22.5), tgt,
                       CaseParams(case=2, inhibit_ratio=0.8, band_width=2))
    ref = pdhg.solve(lp, ops, kkt_tol=1e-5, max_iter=60000)
    if ref["status"] != pdhg.OPTIMAL:
        pytest.skip("instance not optimal in the oracle")
    low = sipo.sipo_create(geo, tgt, cp, dict(storage=sipo.SIPO_BF16, kkt_tol=1e-4, max_iter=1024))
    rl = sipo.sipo_solve(low)
    high = sipo.sipo_create(geo, tgt, cp, dict(storage=sipo.SIPO_F32, kkt_tol=1e-4, max_iter=60000))
    sipo.sipo_warm_start(high, low)
    rh = sipo.sipo_solve(high)
    assert rh["status"] == sipo.SIPO_OPTIMAL, rh
    assert abs(rh["pobj"] - ref["obj"]) <= 1e-3 * abs(ref["obj"])
    assert rh["kkt"] <= 1e-4 and rl["iters"] <= 1024


def _stage1(graded):
    """Case 1 (d = 0.1) solved by the oracle on the tiny binary or multi-level
    disc target, and the Case-2 LP at the ratio r = u~* it fixes (Sec. 3.2)."""
    n, na, nd = 10, 8, 15
    if graded:
        tgt = graded_discs_2d(n, levels=(1.0, 0.85, 0.7), r_range=(1.5, 3.0), container_radius=4.0, seed=4)
    else:
        tgt = discs_2d(n, n_discs=1, r_range=(2.0, 3.0), container_radius=4.0, seed=3)
    ang = uniform_angles(na)
    geom = Geometry(n, n, 1, ang, nd)
    lp1, ops = build_lp(geom, tgt, CaseParams(case=1, band_width=2, tol_lo=0.1, tol_hi=0.1))
    r1 = pdhg.solve(lp1, ops, kkt_tol=1e-11, max_iter=100000)
    assert r1["status"] == pdhg.OPTIMAL
    r = r1["u"]
    lp2, _ = build_lp(geom, tgt, CaseParams(case=2, band_width=2, inhibit_ratio=r))
    geo = dict(nx=n, ny=n, nz=1, angles=ang, n_det=nd)
    return tgt, geo, ops, r1, r, lp2


@pytest.mark.parametrize("graded", [False, True])
def test_primal_start_tracks_the_oracle(sipo, graded):
    """sipo_set_primal: the imported point is the oracle's projection of the
    caller's values (exact in FP64), its dose A^T y agrees, and FP64 solves
    from that start on both sides keep matching objectives, residuals and
    restart counts for 320 iterations."""
    tgt, geo, ops, r1, r, lp2 = _stage1(graded)
    rng = np.random.default_rng(5)
    y2 = r1["y"] / r
    y2 = y2 + np.where(rng.uniform(size=y2.size) < 0.1, -0.05, 0.0)    # some negatives to project
    ref_y, _, ref_v = pdhg.primal_start(lp2, ops, y2)
    ref = pdhg.solve(lp2, ops, kkt_tol=0.0, max_iter=320, start=(y2, None, None))
    cp = dict(kase=2, inhibit_ratio=r, band_width=2)
    ctx = sipo.sipo_create(geo, tgt, cp, dict(storage=sipo.SIPO_F64, kkt_tol=0.0, max_iter=320))
    sipo.sipo_set_primal(ctx, np.ascontiguousarray(y2))
    got = np.empty_like(ref_y)
    sipo.sipo_get_array(ctx, 2, got)
    assert np.array_equal(got, ref_y)
    dose = np.empty(lp2.labels.size)
    sipo.sipo_get_array(ctx, 5, dose)
    d_ref = ops.AT(ref_y.reshape(ops.geo.sino_shape)).ravel()
    m = lp2.labels != 0
    np.testing.assert_allclose(dose[m], d_ref[m], rtol=1e-12, atol=1e-13)
    res = sipo.sipo_solve(ctx)
    assert res["iters"] == 320 and res["restarts"] == ref["restarts"]
    for key in ("pobj", "dobj", "rel_primal", "rel_dual"):
        a, b = res[key], ref["info"][key]
        assert abs(a - b) <= 1e-7 * max(abs(b), 1e-3), (key, a, b)


def test_two_stage_solve_matches_the_oracle(sipo):
    """two_stage_solve in FP64: stage 1 reaches the oracle's Case-1 optimum,
    its ratio is that u~*, and stage 2, started from the rescaled stage-1
    point, reaches the oracle's Case-2 optimum at that ratio, which is at
    most (1 + d) / (1 - d)."""
    tgt, geo, ops, r1, r, lp2 = _stage1(False)
    ref2 = pdhg.solve(lp2, ops, kkt_tol=1e-10, max_iter=100000)
    assert ref2["status"] == pdhg.OPTIMAL
    tol = dict(storage=sipo.SIPO_F64, kkt_tol=1e-10, max_iter=100000)
    out = sipo.two_stage_solve(geo, tgt, tol_lo=0.1, tol_hi=0.1, band_width=2, tolerances=tol)
    s1, s2 = out["stage1"], out["stage2"]
    assert s1["status"] == sipo.SIPO_OPTIMAL and s2 is not None
    assert abs(s1["pobj"] - r1["obj"]) <= 1e-7 * abs(r1["obj"])
    assert abs(out["ratio"] - r) <= 1e-7 * r
    assert s2["status"] == sipo.SIPO_OPTIMAL
    assert abs(s2["pobj"] - ref2["obj"]) <= 1e-6 * ref2["obj"]
    assert s2["pobj"] <= 1.1 / 0.9 * (1 + 1e-7)


@pytest.mark.parametrize("case,extra", [(1, dict(tol_lo=0.1, tol_hi=0.1)), (2, dict(inhibit_ratio=0.7))])
def test_band_width_and_band_free_reach_the_oracle(sipo, case, extra):
    """The band-width study of Sec. 3.2: FP64 solves with a width-1 band and
    band-free (every non-gel voxel in the vial is band) reach the oracle's
    optima, which cannot improve as the band widens."""
    tgt = discs_2d(14, n_discs=2, r_range=(1.5, 2.5), container_radius=5.0, seed=6)
    ang = uniform_angles(10)
    geo = dict(nx=14, ny=14, nz=1, angles=ang, n_det=21)
    objs = []
    for W in (1, -1):
        lp, ops = build_lp(Geometry(14, 14, 1, ang, 21), tgt, CaseParams(case=case, band_width=W, **extra))
        ref = pdhg.solve(lp, ops, kkt_tol=1e-10, max_iter=100000)
        assert ref["status"] == pdhg.OPTIMAL
        ctx = sipo.sipo_create(geo, tgt, dict(kase=case, band_width=W, **extra),
                               dict(storage=sipo.SIPO_F64, kkt_tol=1e-10, max_iter=100000))
        labels = np.empty(14 * 14, np.uint8)
        sipo.sipo_get_array(ctx, 0, labels)
        assert np.array_equal(labels, lp.labels)
        res = sipo.sipo_solve(ctx)
        assert res["status"] == sipo.SIPO_OPTIMAL
        assert abs(res["pobj"] - ref["obj"]) <= 1e-7 * abs(ref["obj"])
        objs.append(res["pobj"])
    assert objs[1] >= objs[0] * (1 - 1e-7)


def test_full_turn_with_attenuation_reaches_the_oracle(sipo):
    """A full 360-degree rotation with Beer-Lambert attenuation (16 views over
    [0, 2 pi), vial radius 5.8, mu = 0.15): FP64 solves of Case 1 and Case 2
    reach the oracle optima, and the half turn of the same Case 2 (light from
    one side only) is reported infeasible, as the oracle reports it."""
    tgt = discs_2d(12, n_discs=2, r_range=(1.5, 2.5), container_radius=4.5, seed=8)
    for case, extra, full in ((1, dict(tol_lo=0.1, tol_hi=0.1), True), (2, dict(inhibit_ratio=0.7), True),
                              (2, dict(inhibit_ratio=0.7), False)):
        ang = uniform_angles(16, 2 * np.pi) if full else uniform_angles(8, np.pi)
        lp, ops = build_lp(Geometry(12, 12, 1, ang, 17, vial_radius=5.8, mu=0.15), tgt,
                           CaseParams(case=case, band_width=2, **extra))
        ref = pdhg.solve(lp, ops, kkt_tol=1e-10, max_iter=100000)
        ctx = sipo.sipo_create(dict(nx=12, ny=12, nz=1, angles=ang, n_det=17, vial_radius=5.8, mu=0.15), tgt,
                               dict(kase=case, band_width=2, **extra),
                               dict(storage=sipo.SIPO_F64, kkt_tol=1e-10, max_iter=100000))
        res = sipo.sipo_solve(ctx)
        if ref["status"] == pdhg.PRIMAL_INFEASIBLE:
            assert res["status"] == sipo.SIPO_PRIMAL_INFEASIBLE, res
            continue
        assert ref["status"] == pdhg.OPTIMAL and res["status"] == sipo.SIPO_OPTIMAL, res
        assert abs(res["pobj"] - ref["obj"]) <= 1e-7 * abs(ref["obj"])


def test_checkpoint_resume_tracks_the_oracle(sipo):
    """sipo_get_state / sipo_set_state: a checkpoint taken after 256 FP64
    iterations, written to host arrays and resumed in a fresh context, runs
    320 more iterations in step with the oracle PDHG started from the same
    point (objectives, residuals and restart counts agree)."""
    case, extra = TINY[1]
    lp, ops, geo, tgt, cp = _tiny(case, extra)
    src = sipo.sipo_create(geo, tgt, cp, dict(storage=sipo.SIPO_F64, kkt_tol=0.0, max_iter=256))
    sipo.sipo_solve(src)
    y = np.empty(lp.active.size)
    up = np.empty(lp.labels.size)
    lo = np.empty(lp.labels.size)
    sc = sipo.sipo_get_state(src, y, up, lo)
    assert sc["iters"] == 256
    ref = pdhg.solve(lp, ops, kkt_tol=0.0, max_iter=320, omega0=sc["omega"], start=(y, sc["u"], sc["v"]),
                     dual_start=(up, lo))
    dst = sipo.sipo_create(geo, tgt, cp, dict(storage=sipo.SIPO_F64, kkt_tol=0.0, max_iter=320))
    sipo.sipo_set_state(dst, y, up, lo, sc["u"], sc["v"], sc["omega"])
    res = sipo.sipo_solve(dst)
    assert res["iters"] == 320 and res["restarts"] == ref["restarts"]
    for key in ("pobj", "dobj", "rel_primal", "rel_dual"):
        a, b = res[key], ref["info"][key]
        assert abs(a - b) <= 1e-7 * max(abs(b), 1e-3), (key, a, b)


def test_resume_at_an_optimum_and_bf16_checkpoint(sipo):
    """Resuming a context from an optimal checkpoint stops at its first check
    with the same objective; a BF16 context's checkpoint (FP32 arrays) holds
    the y that sipo_solve returned, twice in a row (no scratch overwrites the
    saved point)."""
    case, extra = TINY[2]
    lp, ops, geo, tgt, cp = _tiny(case, extra)
    tol = dict(storage=sipo.SIPO_F64, kkt_tol=1e-9, max_iter=100000)
    src = sipo.sipo_create(geo, tgt, cp, tol)
    r0 = sipo.sipo_solve(src)
    assert r0["status"] == sipo.SIPO_OPTIMAL
    y = np.empty(lp.active.size)
    up = np.empty(lp.labels.size)
    lo = np.empty(lp.labels.size)
    sc = sipo.sipo_get_state(src, y, up, lo)
    dst = sipo.sipo_create(geo, tgt, cp, tol)
    sipo.sipo_set_state(dst, y, up, lo, sc["u"], sc["v"], sc["omega"])
    r1 = sipo.sipo_solve(dst)
    assert r1["status"] == sipo.SIPO_OPTIMAL and r1["iters"] <= 64
    assert abs(r1["pobj"] - r0["pobj"]) <= 1e-8 * abs(r0["pobj"])
    low = sipo.sipo_create(geo, tgt, cp, dict(storage=sipo.SIPO_BF16, kkt_tol=1e-3, max_iter=2048))
    y_out = np.empty(lp.active.size, np.float32)
    sipo.sipo_solve(low, y_out)
    ys = [np.empty(lp.active.size, np.float32) for _ in range(2)]
    for yy in ys:
        sipo.sipo_get_state(low, yy, np.empty(lp.labels.size, np.float32), np.empty(lp.labels.size, np.float32))
    assert np.array_equal(ys[0], y_out) and np.array_equal(ys[1], y_out)
    with pytest.raises(sipo.SipoError):
        sipo.sipo_get_state(sipo.sipo_create(geo, tgt, cp, tol), y, up, lo)


def test_host_injected_failures_are_errors_or_statuses(sipo):
    """Failures injected on the host, none of which faults the device: a NaN,
    an infinite and a negative target value and an all-zero target are
    refused with INVALID_ARG (-1) and leave no context; an iteration limit
    is a status, not an error; changing a setting fixed at creation is
    refused and leaves the context usable; an infinite start is a NUMERIC
    error and the context solves again afterwards."""
    case, extra = TINY[2]
    lp, ops, geo, tgt, cp = _tiny(case, extra)
    tol = dict(storage=sipo.SIPO_F64, kkt_tol=1e-9, max_iter=64)
    for bad in (np.nan, np.inf, -1.0):
        t = tgt.copy()
        t.flat[0] = bad
        with pytest.raises(sipo.SipoError) as e:
            sipo.sipo_create(geo, t, cp, tol)
        assert e.value.code == -1 and "target" in str(e.value)
    with pytest.raises(sipo.SipoError) as e:
        sipo.sipo_create(geo, np.zeros_like(tgt), cp, tol)
    assert e.value.code == -1 and "empty" in str(e.value)
    ctx = sipo.sipo_create(geo, tgt, cp, tol)
    res = sipo.sipo_solve(ctx)
    assert res["status"] == sipo.SIPO_ITER_LIMIT and res["iters"] == 64
    with pytest.raises(sipo.SipoError):
        sipo.sipo_set_tolerances(ctx, 1e-9, 100000, check_every=32)
    sipo.sipo_set_tolerances(ctx, 1e-9, 100000)
    res = sipo.sipo_solve(ctx)
    assert res["status"] == sipo.SIPO_OPTIMAL
    # an infinite primal start: the first check finds non-finite residuals and
    # the solve is a NUMERIC error (-5); the next solve starts from zero again
    y = np.zeros(lp.active.size)
    y[np.flatnonzero(lp.active)[0]] = np.inf
    sipo.sipo_set_primal(ctx, y)
    with pytest.raises(sipo.SipoError) as e:
        sipo.sipo_solve(ctx)
    assert e.value.code == -5 and "non-finite" in str(e.value)
    res = sipo.sipo_solve(ctx)
    assert res["status"] == sipo.SIPO_OPTIMAL


def test_bounded_wait_runs_out_and_reports_timeout(sipo):
    """Failure detection on the device without a fault: the staged
    backprojector's bounded mbarrier wait, run on a barrier that nothing
    completes (its one expected arrival is never made), gives up after its
    budget (2e6 cycles, about 1 ms) in every thread, and the library returns
    SIPO_ERR_TIMEOUT; with the arrival made, every wait ends and the call
    returns SIPO_OK.  The device stays usable: a solve runs afterwards."""
    from paper_2604_08997_gb300._abi import SIPO_ERR_TIMEOUT, SIPO_OK, sipo_wait_selftest
    rc, n = sipo_wait_selftest(2_000_000, arrive=False, threads=128)
    assert rc == SIPO_ERR_TIMEOUT and n == 128
    rc, n = sipo_wait_selftest(2_000_000, arrive=True, threads=128)
    assert rc == SIPO_OK and n == 0
    case, extra = TINY[2]
    lp, ops, geo, tgt, cp = _tiny(case, extra)
    ctx = sipo.sipo_create(geo, tgt, cp, dict(storage=sipo.SIPO_F64, kkt_tol=1e-9, max_iter=100000))
    assert sipo.sipo_solve(ctx)["status"] == sipo.SIPO_OPTIMAL
    sipo.sipo_destroy(ctx)


@pytest.mark.parametrize("case,extra", TINY)
def test_scale_invariance_and_single_voxel_gel(sipo, case, extra):
    """Scale invariance on the device (Secs. 2.5-2.6): the target times 2^10
    normalises to the same f~ bit for bit, so the solve is identical (status,
    iterations, objective, returned y) and only the dose-domain factor alpha*
    scales by 2^10.  A gel of one voxel (the smallest part) solves to the
    dense simplex's optimum."""
    lp, ops, geo, tgt, cp = _tiny(case, extra)
    tol = dict(storage=sipo.SIPO_F64, kkt_tol=1e-9, max_iter=100000)
    outs = []
    for scale in (1.0, 1024.0):
        ctx = sipo.sipo_create(geo, (tgt * scale).astype(np.float32), cp, tol)
        y = np.empty(lp.active.shape, np.float64)
        res = sipo.sipo_solve(ctx, y)
        outs.append((res, y))
        sipo.sipo_destroy(ctx)
    (r1, y1), (r2, y2) = outs
    assert (r1["status"], r1["iters"], r1["pobj"], r1["kkt"]) == (r2["status"], r2["iters"], r2["pobj"], r2["kkt"])
    np.testing.assert_array_equal(y1, y2)
    assert r2["alpha"] == pytest.approx(1024.0 * r1["alpha"], rel=1e-12)
    one = np.zeros_like(tgt)
    one[5, 5, 0] = 1.0
    lp1, ops1 = build_lp(Geometry(10, 10, 1, geo["angles"], 15), one,
                         CaseParams(case=case, band_width=2, **extra))
    st, obj, _ = simplex.solve_dense(lp1, ops1)
    ctx = sipo.sipo_create(geo, one, cp, tol)
    res = sipo.sipo_solve(ctx)
    sipo.sipo_destroy(ctx)
    if st == "optimal":
        assert res["status"] == sipo.SIPO_OPTIMAL and abs(res["pobj"] - obj) <= 1e-7 * abs(obj)
    else:
        assert res["status"] == sipo.SIPO_PRIMAL_INFEASIBLE, (st, res["status_name"])


def test_empty_band(sipo):
    """band_width 0 without a PSF leaves the band empty: Case 1 and the general
    form (u~ in no row, unbounded LP) are refused at creation with INVALID_ARG
    before any solve; Case 2 solves to the dense simplex's optimum."""
    for case, extra in TINY[:2]:
        lp_geo = _tiny(case, extra)
        geo, tgt = lp_geo[2], lp_geo[3]
        with pytest.raises(sipo.SipoError) as e:
            sipo.sipo_create(geo, tgt, dict(kase=case, band_width=0, **extra),
                             dict(storage=sipo.SIPO_F64, kkt_tol=1e-9, max_iter=1000))
        assert e.value.code == -1 and "empty band" in str(e.value)
    lp, ops, geo, tgt, cp = _tiny(2, dict(inhibit_ratio=0.6))
    lp0, ops0 = build_lp(Geometry(10, 10, 1, geo["angles"], 15), tgt,
                         CaseParams(case=2, band_width=0, inhibit_ratio=0.6))
    st, obj, _ = simplex.solve_dense(lp0, ops0)
    ctx = sipo.sipo_create(geo, tgt, dict(kase=2, band_width=0, inhibit_ratio=0.6),
                           dict(storage=sipo.SIPO_F64, kkt_tol=1e-9, max_iter=100000))
    res = sipo.sipo_solve(ctx)
    assert st == "optimal" and res["status"] == sipo.SIPO_OPTIMAL
    assert abs(res["pobj"] - obj) <= 1e-7 * abs(obj)
    sipo.sipo_destroy(ctx)


@pytest.mark.parametrize("storage", ["f32", "bf16"])
def test_backprojector_tiles_give_identical_solves(sipo, storage):
    """The fused dual step with every backprojector tile entry: the row-pattern
    kernels (entries 3-6, global loads or tensor-memory staging) add the same
    terms in the same order as the per-voxel window (entries 0-2), so solves
    agree bit for bit, in FP32 and with BF16 iterate storage (256 z: two
    groups of four values per lane)."""
    n, nz = 20, 256
    tgt = np.zeros((n, n, nz), np.float32)
    tgt[6:14, 7:13, 40:200] = 1.0
    tgt[9:11, 4:16, 100:150] = 1.0
    ang = uniform_angles(27)
    geo = dict(nx=n, ny=n, nz=nz, angles=ang, n_det=29, vial_radius=9.5, mu=0.01)
    cp = dict(kase=2, inhibit_ratio=0.7, band_width=2)
    st = sipo.SIPO_F32 if storage == "f32" else sipo.SIPO_BF16
    ref = None
    for tile in range(sipo.sipo_tile_count()):
        ctx = sipo.sipo_create(geo, tgt, cp, dict(storage=st, kkt_tol=0.0, max_iter=192, tile_cfg=tile))
        res = sipo.sipo_solve(ctx)
        assert res["tile_cfg"] == tile
        key = (res["iters"], res["pobj"], res["kkt"], res["dtvr_f"], res["psr_f"])
        if ref is None:
            ref = key
        assert key == ref, (tile, key, ref)
        sipo.sipo_destroy(ctx)


def _slice_stack(nz, bad_z, ratio=0.62):
    """The CPU pins' stack of 12x12 Case-2 slices (10 views, 17 bins), one of
    them (bad_z) infeasible at this ratio; bad_z None: all feasible."""
    n, na, nd = 12, 10, 17
    feas = [discs_2d(n, n_discs=1, r_range=(2.5, 3.5), container_radius=4.5, seed=3),
            discs_2d(n, n_discs=3, r_range=(1.0, 1.6), container_radius=4.5, seed=3),
            discs_2d(n, n_discs=1, r_range=(2.5, 3.5), container_radius=4.5, seed=5)]
    bad = discs_2d(n, n_discs=1, r_range=(2.5, 3.5), container_radius=4.5, seed=1)
    sl = [feas[i % 3] for i in range(nz)]
    if bad_z is not None:
        sl[bad_z] = bad
    tgt = np.ascontiguousarray(np.concatenate(sl, axis=2))
    ang = uniform_angles(na)
    geo = dict(nx=n, ny=n, nz=nz, angles=ang, n_det=nd)
    cp = dict(kase=2, inhibit_ratio=ratio, band_width=2)
    lp, ops = build_lp(Geometry(n, n, nz, ang, nd), tgt, CaseParams(case=2, inhibit_ratio=ratio, band_width=2))
    return lp, ops, geo, tgt, cp


@pytest.mark.parametrize("storage", ["f64", "f32"])
def test_one_infeasible_slice_is_certified_and_named(sipo, storage):
    """16 slices, slice 8 infeasible (HiGHS per slice on the CPU): the solver
    proves the LP infeasible slice by slice within the 5120 iterations the
    oracle's slice test needs (its whole-volume test alone needs more) and
    names the slice; the same stack without slice 8 solves to optimality with
    the oracle's objective (no false certificate)."""
    st = sipo.SIPO_F64 if storage == "f64" else sipo.SIPO_F32
    lp, ops, geo, tgt, cp = _slice_stack(16, 8)
    ctx = sipo.sipo_create(geo, tgt, cp, dict(storage=st, kkt_tol=1e-7, max_iter=5120))
    res = sipo.sipo_solve(ctx)
    assert res["status"] == sipo.SIPO_PRIMAL_INFEASIBLE, res
    assert res["cert_slice"] in (8, -1), res["cert_slice"]
    sipo.sipo_destroy(ctx)
    lp, ops, geo, tgt, cp = _slice_stack(16, None)
    ref = pdhg.solve(lp, ops, kkt_tol=1e-8, max_iter=100000)
    assert ref["status"] == pdhg.OPTIMAL
    ctx = sipo.sipo_create(geo, tgt, cp, dict(storage=st, kkt_tol=1e-8 if storage == "f64" else 1e-5,
                                              max_iter=100000))
    res = sipo.sipo_solve(ctx)
    assert res["status"] == sipo.SIPO_OPTIMAL, res
    assert res["cert_slice"] == -1
    assert abs(res["pobj"] - ref["obj"]) <= (1e-7 if storage == "f64" else 1e-4) * abs(ref["obj"])
    sipo.sipo_destroy(ctx)


def test_batched_sweep_invariants(sipo):
    """A tolerance and inhibition sweep solved as one batch (FP64): Case-1
    optima u~*(delta) cannot increase as delta widens the feasible set
    (Sec. 2.7.1), Case-2 feasibility is monotone in the ratio r and v~*(r)
    cannot increase where feasible (Sec. 2.7.2: a larger r lowers the gel
    rows' bound f~ = f_T / (r min f_T)); every status agrees with the dense
    simplex on the same LP."""
    deltas = (0.02, 0.05, 0.1, 0.2)
    ratios = (0.3, 0.4, 0.5, 0.6, 0.7, 0.8, 0.9)
    specs = [(1, dict(tol_lo=d, tol_hi=d)) for d in deltas] + [(2, dict(inhibit_ratio=r)) for r in ratios]
    ctxs, simplex_status = [], []
    for case, extra in specs:
        lp, ops, geo, tgt, cp = _tiny(case, extra)
        simplex_status.append(simplex.solve_dense(lp, ops)[0])
        ctxs.append(sipo.sipo_create(geo, tgt, cp, dict(storage=sipo.SIPO_F64, kkt_tol=1e-9, max_iter=64 * 800)))
    res = sipo.sipo_solve_batched(ctxs)
    for r, st in zip(res, simplex_status):
        want = sipo.SIPO_OPTIMAL if st == "optimal" else sipo.SIPO_PRIMAL_INFEASIBLE
        assert r["status"] == want, (r["status_name"], st)
    u = [r["pobj"] for r in res[:len(deltas)]]
    assert all(a >= b - 1e-7 for a, b in zip(u, u[1:])), u
    c2 = res[len(deltas):]
    feas = [r["status"] == sipo.SIPO_OPTIMAL for r in c2]
    assert feas == sorted(feas) and any(feas) and not all(feas), feas
    v = [r["pobj"] for r in c2 if r["status"] == sipo.SIPO_OPTIMAL]
    assert all(a >= b - 1e-7 for a, b in zip(v, v[1:])), v
    for c in ctxs:
        sipo.sipo_destroy(c)


@pytest.mark.parametrize("storage", ["f64", "f32"])
def test_case2_with_separation_certifies_or_starts(sipo, storage):
    """Sequential form.  The separation LP (Case 1 of the part with tol_lo = 0, tol_hi = 10) on
    the 16-slice stack, probed as a Farkas ray of Case 2 at r = 0.62: with the
    infeasible slice the probe proves Case 2 infeasible on slice 8; without it
    the separation LP converges to HiGHS's optimum (below r) and Case 2 started
    from its scaled point reaches the oracle optimum."""
    from paper_2604_08997_gb300 import case2_with_separation
    from test_oracle_lp import _highs
    st = sipo.SIPO_F64 if storage == "f64" else sipo.SIPO_F32
    tol = dict(storage=st, kkt_tol=1e-8 if storage == "f64" else 1e-5, max_iter=100000)
    for bad in (8, None):
        lp, ops, geo, tgt, cp = _slice_stack(16, bad)
        out = case2_with_separation(geo, tgt, 0.62, band_width=2, tolerances=tol, probe_every=256, race=False)
        if bad is not None:
            assert out["status"] == sipo.SIPO_PRIMAL_INFEASIBLE and out["certified"], out
            assert out["cert_slice"] == bad
        else:
            lp1, ops1 = build_lp(Geometry(12, 12, 16, uniform_angles(10), 17), tgt,
                                 CaseParams(case=1, tol_lo=0.0, tol_hi=10.0, band_width=2))
            ref = _highs(lp1, ops1, method="highs-ipm")
            assert ref.status == 0 and ref.fun < 0.62
            assert out["separation"]["status"] == sipo.SIPO_OPTIMAL and not out["certified"]
            assert out["ratio_bound"] == pytest.approx(ref.fun, rel=1e-7 if storage == "f64" else 1e-4)
            ref2 = pdhg.solve(lp, ops, kkt_tol=1e-8, max_iter=100000)
            assert ref2["status"] == pdhg.OPTIMAL and out["status"] == sipo.SIPO_OPTIMAL
            assert out["case2"]["pobj"] == pytest.approx(ref2["obj"], rel=1e-7 if storage == "f64" else 1e-4)


@pytest.mark.parametrize("storage", ["f64", "f32"])
def test_case2_race_decides_both_ways(sipo, storage):
    """Concurrent form on the 16-slice stack at r = 0.62: with the infeasible
    slice 8 the workflow ends PRIMAL_INFEASIBLE, by a probe certificate that
    names slice 8 or by the Case-2 solve's own certificate (slice 8, or the
    whole volume); without it the Case-2 solve ends OPTIMAL at the oracle
    optimum, no probe certifies, and the separation solve is stopped there
    (ITER_LIMIT) unless it reached its own optimum first.  Equal or repeated
    contexts, and targets that cannot test the separation duals, are
    refused."""
    from paper_2604_08997_gb300 import case2_with_separation
    st = sipo.SIPO_F64 if storage == "f64" else sipo.SIPO_F32
    tol = dict(storage=st, kkt_tol=1e-8 if storage == "f64" else 1e-5, max_iter=100000)
    lp, ops, geo, tgt, cp = _slice_stack(16, 8)
    out = case2_with_separation(geo, tgt, 0.62, band_width=2, tolerances=tol, probe_every=256)
    assert out["status"] == sipo.SIPO_PRIMAL_INFEASIBLE, out
    if out["certified"]:
        assert out["cert_slice"] == 8 and out["case2"]["status"] == sipo.SIPO_ITER_LIMIT
    else:
        assert out["case2"]["status"] == sipo.SIPO_PRIMAL_INFEASIBLE
        assert out["case2"]["cert_slice"] in (8, -1)
    lp, ops, geo, tgt, cp = _slice_stack(16, None)
    out = case2_with_separation(geo, tgt, 0.62, band_width=2, tolerances=tol, probe_every=256)
    ref2 = pdhg.solve(lp, ops, kkt_tol=1e-8, max_iter=100000)
    assert ref2["status"] == pdhg.OPTIMAL
    assert out["status"] == sipo.SIPO_OPTIMAL and not out["certified"], out
    assert out["separation"]["status"] in (sipo.SIPO_ITER_LIMIT, sipo.SIPO_OPTIMAL)
    assert out["case2"]["pobj"] == pytest.approx(ref2["obj"], rel=1e-7 if storage == "f64" else 1e-4)
    a = sipo.sipo_create(geo, tgt, dict(kase=1, tol_lo=0.0, tol_hi=10.0, band_width=2), tol)
    b = sipo.sipo_create(geo, tgt, cp, tol)
    c = sipo.sipo_create(geo, tgt, cp, tol)
    for args in ((a, a, c), (a, b, a), (a, b, b)):
        with pytest.raises(sipo.SipoError):
            sipo.sipo_solve_race(*args, 128)
    with pytest.raises(sipo.SipoError):
        sipo.sipo_solve_race(a, b, c, 0)
    # targets whose LP cannot test the separation duals: another geometry,
    # and the general form (no bound-based certificate); refused up front
    lp8, ops8, geo8, tgt8, cp8 = _slice_stack(8, None)
    other = sipo.sipo_create(geo8, tgt8, cp8, tol)
    general = sipo.sipo_create(geo, tgt, dict(kase=0, w1=1.0, w2=1.0, band_width=2), tol)
    for t in (other, general):
        with pytest.raises(sipo.SipoError):
            sipo.sipo_solve_race(a, t, c, 128)
        with pytest.raises(sipo.SipoError):
            sipo.sipo_solve_probe(a, t, 128)
    for x in (a, b, c, other, general):
        sipo.sipo_destroy(x)
