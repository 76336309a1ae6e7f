"""Pins for the oracle LP and PDHG (CPU only).

The PDHG oracle is checked against exact LP optima (a dense simplex with
Bland's rule, and scipy's HiGHS as an independent library routine), against
the KKT stationarity conditions of Sec. 6.1 (Eqs. 48-49), against the exactness
of the Charnes-Cooper transform (Sec. 2.6.2: the LP optimum equals the
fractional objective of its solution), against scale invariance (Secs. 2.5 and
2.6.2) and against the closed-form post-scaling factor (Eq. 27).
"""
import math

import numpy as np
import pytest
import scipy.sparse as sp
from scipy.optimize import linprog, minimize_scalar

from oracle import pdhg, simplex
from oracle.lp import (BAND, CASE1, CASE2, EXT, GEL, GENERAL, CaseParams, build_lp,
                       metrics, partition)
from oracle.operators import Geometry
from synthetic.targets import discs_2d, graded_discs_2d, uniform_angles

TINY = [
    (GENERAL, {}),
    (CASE1, dict(tol_lo=0.1, tol_hi=0.1)),
    (CASE2, dict(inhibit_ratio=0.6)),
]


def _tiny(case, extra, n=10, na=8, nd=15, seed=3, scale=1.0):
    tgt = discs_2d(n, n_discs=1, r_range=(2.0, 3.0), container_radius=4.0, seed=seed) * scale
    geo = Geometry(n, n, 1, uniform_angles(na), nd)
    return build_lp(geo, tgt, CaseParams(case=case, band_width=2, **extra))


@pytest.fixture(scope="module")
def tiny_solutions():
    out = {}
    for case, extra in TINY:
        lp, ops = _tiny(case, extra)
        st, obj, _ = simplex.solve_dense(lp, ops)
        res = pdhg.solve(lp, ops, kkt_tol=1e-10, max_iter=60000)
        out[case] = (lp, ops, st, obj, res)
    return out


def test_partition_single_voxel():
    f = np.zeros((9, 9, 1))
    f[4, 4, 0] = 1.0
    geo = Geometry(9, 9, 1, np.zeros(1), 9)
    lab = partition(geo, f, 2)
    assert (lab == GEL).sum() == 1
    # lattice points with 0 < a^2 + b^2 <= 4
    assert (lab == BAND).sum() == 12
    assert (partition(geo, f, 0) == BAND).sum() == 0
    assert (partition(geo, f, -1) == BAND).sum() == 80
    geo_k = Geometry(9, 9, 1, np.zeros(1), 9, psf_sigma=(0.25, 0.25, 0.0))  # radius 1
    assert (partition(geo_k, f, 0) == BAND).sum() == 8
    geo_v = Geometry(9, 9, 1, np.zeros(1), 9, vial_radius=1.2)
    lab_v = partition(geo_v, f, 2)
    assert (lab_v == BAND).sum() == 4 and (lab_v == EXT).sum() == 76


@pytest.mark.parametrize("case", [GENERAL, CASE1, CASE2])
def test_pdhg_matches_dense_simplex(tiny_solutions, case):
    lp, ops, st, obj, res = tiny_solutions[case]
    assert st == "optimal"
    assert res["status"] == pdhg.OPTIMAL
    assert abs(res["obj"] - obj) <= 1e-7 * abs(obj)


@pytest.mark.parametrize("case", [GENERAL, CASE1, CASE2])
def test_kkt_stationarity_and_cct_exactness(tiny_solutions, case):
    """Eqs. 48-49 at the optimum; the recovered scale s = min_gel(d / f~) = 1 (t = 1/s,
    Eq. 18) and the fractional objective of y* equals the LP objective (Sec. 2.6.2)."""
    lp, ops, st, obj, res = tiny_solutions[case]
    info, m = res["info"], res["metrics"]
    # with the implied bounds u~ >= 0, v~ >= 1 a bound multiplier takes up the
    # slack when the bound is active; otherwise Eqs. 48-49 hold as printed
    if lp.has_u:
        if res["u"] > 1e-6:
            assert abs(info["S_band"] - lp.c_u) < 1e-6
        else:
            assert info["S_band"] <= lp.c_u + 1e-6
    if lp.has_v:
        if res["v"] > 1.0 + 1e-6:
            assert abs(info["S_gel"] - lp.c_v) < 1e-6
        else:
            assert info["S_gel"] <= lp.c_v + 1e-6
    assert abs(m["s"] - 1.0) < 1e-6
    frac = 0.0
    if lp.has_u:
        frac += lp.c_u * m["band_max"]
    if lp.has_v:
        frac += lp.c_v * m["gel_max_ratio"]
    if not lp.has_u and not lp.has_v:
        pytest.skip("no objective")
    assert abs(frac - obj) <= 1e-6 * abs(obj)
    if case == CASE2:
        assert abs(m["dtvr_f"] - obj) <= 1e-6 * obj      # DTVR(y*) = v~* when min ratio = 1


def test_infeasible_case2_reported_by_both():
    lp, ops = _tiny(CASE2, dict(inhibit_ratio=0.3))
    st, _, _ = simplex.solve_dense(lp, ops)
    assert st == "infeasible"
    res = pdhg.solve(lp, ops, kkt_tol=1e-9, max_iter=20000)
    assert res["status"] == pdhg.PRIMAL_INFEASIBLE


def _highs(lp, ops, method="highs"):
    """The LP of `lp` for scipy's HiGHS (no PSF): the slice operator P^T on
    every z-slice, i.e. P^T (x) I_nz in the [y][x][z] / [angle][bin][z] order."""
    assert not any(s > 0 for s in ops.geo.psf_sigma)
    act = np.flatnonzero(lp.active)
    PT = ops.PT if ops.geo.nz == 1 else sp.kron(ops.PT, sp.identity(ops.geo.nz), format="csr")
    M = PT[:, act]
    band, gel = np.flatnonzero(lp.band), np.flatnonzero(lp.gel)
    nb, ng, ny = band.size, gel.size, act.size
    ucol = sp.csr_matrix((-np.ones(nb) if lp.has_u else np.zeros(nb),
                          (np.arange(nb), np.zeros(nb, int))), shape=(nb, 1))
    vcol = sp.csr_matrix((-lp.ft[gel] if lp.has_v else np.zeros(ng),
                          (np.arange(ng), np.zeros(ng, int))), shape=(ng, 1))
    zb, zg = sp.csr_matrix((nb, 1)), sp.csr_matrix((ng, 1))
    G = sp.vstack([sp.hstack([M[band], ucol, zb]), sp.hstack([M[gel], zg, vcol]),
                   sp.hstack([-M[gel], zg, zg])]).tocsr()
    h = np.concatenate([np.zeros(nb) if lp.has_u else np.ones(nb),
                        np.zeros(ng) if lp.has_v else lp.upper[gel], -lp.lower[gel]])
    c = np.zeros(ny + 2)
    c[ny] = lp.c_u if lp.has_u else 0.0
    c[ny + 1] = lp.c_v if lp.has_v else 0.0
    bounds = [(0, None)] * ny + [(None, None) if lp.has_u else (0, 0),
                                 (None, None) if lp.has_v else (0, 0)]
    res = linprog(c, A_ub=G, b_ub=h, bounds=bounds, method=method)
    return res


@pytest.mark.parametrize("case,extra", [(CASE1, dict(tol_lo=0.05, tol_hi=0.05)),
                                        (CASE2, dict(inhibit_ratio=0.7))])
def test_pdhg_matches_highs_on_small_slice(case, extra):
    tgt = discs_2d(24, n_discs=2, r_range=(3.0, 5.0), container_radius=10.0, seed=11)
    geo = Geometry(24, 24, 1, uniform_angles(32), 35)
    lp, ops = build_lp(geo, tgt, CaseParams(case=case, band_width=3, **extra))
    ref = _highs(lp, ops)
    assert ref.status == 0
    res = pdhg.solve(lp, ops, kkt_tol=1e-8, max_iter=40000)
    assert res["status"] == pdhg.OPTIMAL
    assert abs(res["obj"] - ref.fun) <= 1e-6 * abs(ref.fun)


def _physical_highs(f_T, case, extra, ops, labels, active):
    """The projection LP written in dose units straight from the case
    definitions (Sec. 2.6.2 general form, Sec. 2.7.1 Case 1, Sec. 2.7.2 Case 2),
    with none of the oracle's normalisation by f_crit:

    - general: min w1 u + w2 v, f_T <= f <= v f_T on gel, f <= u min f_T on band;
    - Case 1:  min u, (1 - d_lo) f_T <= f <= (1 + d_hi) f_T on gel,
               f <= u (1 - d_lo) min f_T on band;
    - Case 2:  min v, f_T <= f <= v f_T on gel, f <= r min f_T on band;

    with f = P^T y over the active rays and y >= 0.  The objective is a ratio
    of doses, so it equals the normalised LP's optimum (Sec. 2.5)."""
    fT = np.asarray(f_T, np.float64).ravel()
    act = np.flatnonzero(active)
    M = ops.PT[:, act]
    gel, band = np.flatnonzero(labels == GEL), np.flatnonzero(labels == BAND)
    fmin = fT[gel].min()
    ny, nb, ng = act.size, band.size, gel.size
    if case == CASE1:
        lo, hi = (1 - extra["tol_lo"]) * fT[gel], (1 + extra["tol_hi"]) * fT[gel]
        scale_u = (1 - extra["tol_lo"]) * fmin
    else:
        lo, hi = fT[gel], None
        scale_u = fmin
    # columns: y (ny), u, v
    col = lambda vals, n: sp.csr_matrix((vals, (np.arange(n), np.zeros(n, int))), shape=(n, 1))
    zb, zg = sp.csr_matrix((nb, 1)), sp.csr_matrix((ng, 1))
    if case == CASE2:
        band_blk = sp.hstack([M[band], zb, zb])
        band_rhs = np.full(nb, extra["inhibit_ratio"] * fmin)
    else:
        band_blk = sp.hstack([M[band], col(-np.full(nb, scale_u), nb), zb])
        band_rhs = np.zeros(nb)
    if case == CASE1:
        up_blk, up_rhs = sp.hstack([M[gel], zg, zg]), hi
    else:
        up_blk, up_rhs = sp.hstack([M[gel], zg, col(-fT[gel], ng)]), np.zeros(ng)
    G = sp.vstack([band_blk, up_blk, sp.hstack([-M[gel], zg, zg])]).tocsr()
    h = np.concatenate([band_rhs, up_rhs, -lo])
    c = np.zeros(ny + 2)
    if case == GENERAL:
        c[ny], c[ny + 1] = 1.0, 1.0
    elif case == CASE1:
        c[ny] = 1.0
    else:
        c[ny + 1] = 1.0
    bounds = [(0, None)] * ny + [(0, None) if case != CASE2 else (0, 0),
                                 (0, None) if case != CASE1 else (0, 0)]
    return linprog(c, A_ub=G, b_ub=h, bounds=bounds, method="highs")


# (levels, seed, case, params): one response level per disc; the Case-2 ratio
# sits below the instance's feasibility threshold (about 0.80 for the first
# target, 0.95 for the second).
GRAY = [((1.0, 0.85, 0.7), 4, GENERAL, {}),
        ((1.0, 0.85, 0.7), 4, CASE1, dict(tol_lo=0.1, tol_hi=0.1)),
        ((1.0, 0.85, 0.7), 4, CASE2, dict(inhibit_ratio=0.9)),
        ((1.0, 0.6, 0.8), 5, GENERAL, {}),
        ((1.0, 0.6, 0.8), 5, CASE1, dict(tol_lo=0.1, tol_hi=0.1)),
        ((1.0, 0.6, 0.8), 5, CASE2, dict(inhibit_ratio=1.0))]


def _gray(levels, seed, case, extra):
    tgt = graded_discs_2d(10, levels=levels, r_range=(1.5, 3.0), container_radius=4.0, seed=seed)
    geo = Geometry(10, 10, 1, uniform_angles(8), 15)
    lp, ops = build_lp(geo, tgt, CaseParams(case=case, band_width=2, **extra))
    return tgt, lp, ops


@pytest.mark.parametrize("levels,seed,case,extra", GRAY)
def test_grayscale_target_matches_dose_unit_lp(levels, seed, case, extra):
    """Multi-level targets (Sec. 3.3: one prescribed level per part): HiGHS on
    the oracle's normalised LP and on the LP written in dose units from the
    definitions give one optimum, and the oracle PDHG reaches it.  A
    normalisation that treated the target as binary, or divided by the wrong
    f_crit, moves the first away from the second."""
    tgt, lp, ops = _gray(levels, seed, case, extra)
    assert np.unique(lp.ft[lp.gel]).size == 3
    ref = _physical_highs(tgt, case, extra, ops, lp.labels, lp.active)
    assert ref.status == 0
    nrm = _highs(lp, ops)
    assert nrm.status == 0
    assert abs(nrm.fun - ref.fun) <= 1e-9 * abs(ref.fun)
    res = pdhg.solve(lp, ops, kkt_tol=1e-10, max_iter=80000)
    assert res["status"] == pdhg.OPTIMAL
    assert abs(res["obj"] - ref.fun) <= 1e-8 * abs(ref.fun)
    assert abs(metrics(lp, res["d"])["s"] - 1.0) < 1e-7


def test_grayscale_case2_below_threshold_is_infeasible():
    """Below the feasibility threshold both LP forms are infeasible for HiGHS
    and the oracle PDHG reports Case 2 infeasible on the multi-level target."""
    extra = dict(inhibit_ratio=0.7)
    tgt, lp, ops = _gray((1.0, 0.85, 0.7), 4, CASE2, extra)
    assert _physical_highs(tgt, CASE2, extra, ops, lp.labels, lp.active).status == 2
    assert _highs(lp, ops).status == 2
    res = pdhg.solve(lp, ops, kkt_tol=1e-9, max_iter=40000)
    assert res["status"] == pdhg.PRIMAL_INFEASIBLE


def test_simplex_refuses_a_vertex_off_the_feasible_set():
    """On a multi-level target a pivot on a near-zero tableau entry drives the
    dense simplex off the feasible set; it must raise, not report that
    vertex's objective as the optimum (HiGHS gives the true one)."""
    _, lp, ops = _gray((1.0, 0.6, 0.8), 5, GENERAL, {})
    try:
        st, obj, _ = simplex.solve_dense(lp, ops)
    except RuntimeError as e:
        assert "feasibility" in str(e)
        return
    assert abs(obj - _highs(lp, ops).fun) <= 1e-8 * abs(obj)


def _two_stage_instance(graded):
    if graded:
        tgt = graded_discs_2d(10, levels=(1.0, 0.85, 0.7), r_range=(1.5, 3.0), container_radius=4.0, seed=4)
    else:
        tgt = discs_2d(10, n_discs=1, r_range=(2.0, 3.0), container_radius=4.0, seed=3)
    return tgt, Geometry(10, 10, 1, uniform_angles(8), 15)


@pytest.mark.parametrize("graded", [False, True])
def test_two_stage_case2_at_the_case1_bound(graded):
    """Two-stage design (Sec. 3.2): the Case-1 optimum u~* fixes the inhibition
    ratio r = u~* of a Case-2 solve.  The Case-1 point in Case-2 units,
    y1 / r, satisfies every Case-2 row (gel d >= f~_T, band d <= 1), so the
    Case-2 optimum v~* (HiGHS) is at most its spread, itself at most
    (1 + d_hi) / (1 - d_lo); the oracle PDHG reaches v~* both from zero and
    from that point (its primal start)."""
    delta = 0.1
    tgt, geo = _two_stage_instance(graded)
    lp1, ops = build_lp(geo, tgt, CaseParams(case=CASE1, band_width=2, tol_lo=delta, tol_hi=delta))
    r1 = pdhg.solve(lp1, ops, kkt_tol=1e-11, max_iter=100000)
    assert r1["status"] == pdhg.OPTIMAL
    ref1 = _highs(lp1, ops)
    assert abs(r1["u"] - ref1.fun) <= 1e-8 * ref1.fun
    r = r1["u"]
    lp2, _ = build_lp(geo, tgt, CaseParams(case=CASE2, band_width=2, inhibit_ratio=r))
    y2 = r1["y"] / r
    d2 = ops.AT(y2.reshape(geo.sino_shape)).ravel()
    assert d2[lp2.band].max() <= 1.0 + 1e-8
    assert np.all(d2[lp2.gel] >= lp2.ft[lp2.gel] * (1.0 - 1e-8))
    spread = float(np.max(d2[lp2.gel] / lp2.ft[lp2.gel]))
    assert spread <= (1 + delta) / (1 - delta) * (1 + 1e-8)
    ref2 = _highs(lp2, ops)
    assert ref2.status == 0
    assert ref2.fun <= spread * (1 + 1e-9)
    _, u0, v0 = pdhg.primal_start(lp2, ops, y2)
    assert abs(v0 - spread) <= 1e-12 * spread
    for start in (None, (y2, None, None)):
        res = pdhg.solve(lp2, ops, kkt_tol=1e-10, max_iter=100000, start=start)
        assert res["status"] == pdhg.OPTIMAL
        assert abs(res["obj"] - ref2.fun) <= 1e-8 * ref2.fun


def test_primal_start_projects_onto_the_primal_domain():
    """primal_start zeroes negative, NaN and inactive-ray entries and keeps the
    rest; explicit admissible scalars are kept, inadmissible ones replaced by
    the smallest admissible (v~ >= 1 and v~ f~ >= A^T y on gel)."""
    tgt, geo = _two_stage_instance(False)
    lp, ops = build_lp(geo, tgt, CaseParams(case=GENERAL, band_width=2))
    rng = np.random.default_rng(7)
    y = rng.normal(size=lp.active.size)
    y[3] = np.nan
    yp, u, v = pdhg.primal_start(lp, ops, y, 0.25, -1.0)
    keep = lp.active & np.nan_to_num(y > 0)
    assert np.array_equal(yp[keep], y[keep]) and np.all(yp[~keep] == 0.0)
    assert u == 0.25
    d = ops.AT(yp.reshape(geo.sino_shape)).ravel()
    assert v >= 1.0 and np.all(d[lp.gel] <= v * lp.ft[lp.gel] * (1 + 1e-12))
    assert v == 1.0 or np.any(np.isclose(d[lp.gel], v * lp.ft[lp.gel], rtol=1e-12))


def _band_instance(case, extra, W):
    tgt = discs_2d(14, n_discs=2, r_range=(1.5, 2.5), container_radius=5.0, seed=6)
    geo = Geometry(14, 14, 1, uniform_angles(10), 21)
    return build_lp(geo, tgt, CaseParams(case=case, band_width=W, **extra))


@pytest.mark.parametrize("case,extra", [(GENERAL, {}), (CASE1, dict(tol_lo=0.1, tol_hi=0.1)),
                                        (CASE2, dict(inhibit_ratio=0.7))])
def test_band_width_study_is_monotone(case, extra):
    """Band-region definition (Sec. 3.2): a wider band adds band rows, so the
    band sets are nested (width 1, 2, 3, band-free) and the optimum (HiGHS)
    cannot improve; the oracle PDHG reaches the band-free optimum."""
    prev_band, prev_obj = None, -np.inf
    for W in (1, 2, 3, -1):
        lp, ops = _band_instance(case, extra, W)
        if prev_band is not None:
            assert np.all(lp.band[prev_band]) and lp.band.sum() > prev_band.sum()
        ref = _highs(lp, ops)
        assert ref.status == 0
        assert ref.fun >= prev_obj - 1e-9 * abs(ref.fun)
        prev_band, prev_obj = lp.band.copy(), ref.fun
    res = pdhg.solve(lp, ops, kkt_tol=1e-10, max_iter=100000)
    assert res["status"] == pdhg.OPTIMAL
    assert abs(res["obj"] - ref.fun) <= 1e-8 * abs(ref.fun)


def _turn_instance(case, extra, full, mu):
    tgt = discs_2d(12, n_discs=2, r_range=(1.5, 2.5), container_radius=4.5, seed=8)
    ang = uniform_angles(16, 2 * math.pi) if full else uniform_angles(8, math.pi)
    geo = Geometry(12, 12, 1, ang, 17, vial_radius=5.8, mu=mu)
    return build_lp(geo, tgt, CaseParams(case=case, band_width=2, **extra))


@pytest.mark.parametrize("case,extra", [(GENERAL, {}), (CASE1, dict(tol_lo=0.1, tol_hi=0.1)),
                                        (CASE2, dict(inhibit_ratio=0.7))])
def test_full_turn_against_half_turn(case, extra):
    """A full 360-degree rotation (Sec. 3.1 uses 1-degree steps over a full
    turn).  Without attenuation the view at theta + pi mirrors the one at
    theta (u -> n_det - 1 - u), so 2N views over [0, 2 pi) reach exactly the
    optimum of N views over [0, pi) (the LP is scale invariant).  With
    attenuation the far side is dimmer, the full turn holds every half-turn
    ray and more, and its optimum cannot be worse (here Case 2 turns from
    infeasible to feasible); the oracle PDHG reaches the full-turn optimum."""
    half = _highs(*_turn_instance(case, extra, False, 0.0))
    full = _highs(*_turn_instance(case, extra, True, 0.0))
    assert half.status == 0 and full.status == 0
    assert abs(full.fun - half.fun) <= 1e-9 * abs(half.fun)
    half = _highs(*_turn_instance(case, extra, False, 0.15))
    lp, ops = _turn_instance(case, extra, True, 0.15)
    full = _highs(lp, ops)
    assert full.status == 0
    if case == CASE2:
        assert half.status == 2
    else:
        assert half.status == 0 and full.fun < half.fun * (1 - 1e-3)
    res = pdhg.solve(lp, ops, kkt_tol=1e-10, max_iter=100000)
    assert res["status"] == pdhg.OPTIMAL
    assert abs(res["obj"] - full.fun) <= 1e-8 * abs(full.fun)


def test_resume_from_an_optimal_checkpoint_stops_at_once():
    """Checkpoint and resume: restarting the oracle from its own returned point
    T(z) (y, lam_up, lam_lo, u~, v~, omega) of a solve at KKT 1e-10 stops at
    the first check with the same objective; dual_point keeps an admissible
    dual point and zeroes the rest."""
    lp, ops = _tiny(CASE1, dict(tol_lo=0.1, tol_hi=0.1))
    res = pdhg.solve(lp, ops, kkt_tol=1e-10, max_iter=100000)
    assert res["status"] == pdhg.OPTIMAL
    up, lo = pdhg.dual_point(lp, res["lam_up"], res["lam_lo"])
    assert np.array_equal(up, res["lam_up"]) and np.array_equal(lo, res["lam_lo"])
    junk = np.full(lp.labels.size, -1.0)
    up2, lo2 = pdhg.dual_point(lp, np.abs(junk), np.abs(junk))
    assert np.all(up2[~(lp.band | lp.gel)] == 0) and np.all(lo2[~lp.gel] == 0)
    assert np.all(pdhg.dual_point(lp, junk, junk)[0] == 0)
    again = pdhg.solve(lp, ops, kkt_tol=1e-10, max_iter=100000, omega0=res["omega"],
                       start=(res["y"], res["u"], res["v"]), dual_start=(res["lam_up"], res["lam_lo"]))
    assert again["status"] == pdhg.OPTIMAL and again["iters"] == 0
    # one more step from a point at KKT 1e-10 moves the objective within that tolerance
    assert abs(again["obj"] - res["obj"]) <= 1e-9 * abs(res["obj"])


def test_scale_invariance_bitwise_and_general():
    """f_T -> 2^k f_T leaves the normalised LP and the iterates bitwise unchanged;
    a general factor leaves the optimum unchanged (Sec. 2.5, Eq. 18)."""
    for case, extra in TINY:
        lp1, ops1 = _tiny(case, extra)
        lp2, ops2 = _tiny(case, extra, scale=8.0)
        for name in ("ft", "lower", "upper", "labels", "active"):
            assert np.array_equal(getattr(lp1, name), getattr(lp2, name)), name
        r1 = pdhg.solve(lp1, ops1, kkt_tol=0.0, max_iter=300)
        r2 = pdhg.solve(lp2, ops2, kkt_tol=0.0, max_iter=300)
        assert np.array_equal(r1["y"], r2["y"])
        assert r1["obj"] == r2["obj"]
    lp3, ops3 = _tiny(CASE2, dict(inhibit_ratio=0.6), scale=3.7)
    r3 = pdhg.solve(lp3, ops3, kkt_tol=1e-10, max_iter=60000)
    lp1, ops1 = _tiny(CASE2, dict(inhibit_ratio=0.6))
    r1 = pdhg.solve(lp1, ops1, kkt_tol=1e-10, max_iter=60000)
    assert abs(r3["obj"] - r1["obj"]) < 1e-8


def test_metrics_zero_homogeneous(tiny_solutions):
    lp, ops, _, _, res = tiny_solutions[GENERAL]
    m1 = metrics(lp, res["d"])
    m2 = metrics(lp, 7.3 * res["d"])
    for key in ("dtvr_f", "dsr", "psr_f"):
        assert abs(m1[key] - m2[key]) <= 1e-12 * abs(m1[key])


def test_post_scaling_closed_form(tiny_solutions):
    """Eq. 27: alpha* = <f~*, f_T> / <f~*, f~*> minimises Phi_f; Case 2 gives alpha* <= f_crit."""
    for case in (GENERAL, CASE2):
        lp, ops, _, _, res = tiny_solutions[case]
        d = res["d"]
        gel = lp.gel
        phi = lambda a: np.sum((a * d[gel] - lp.f_T[gel]) ** 2)
        brute = minimize_scalar(phi, bounds=(1e-6, 10.0), method="bounded",
                                options=dict(xatol=1e-12)).x
        assert abs(res["metrics"]["alpha"] - brute) < 1e-6
        if case == CASE2:
            assert res["metrics"]["alpha"] <= lp.f_crit * (1 + 1e-9)


def test_case1_objective_monotone_in_tolerance():
    """Widening the Case-1 tolerance grows the feasible set, so u~*(delta) cannot increase."""
    objs = []
    for delta in (0.05, 0.1, 0.2):
        lp, ops = _tiny(CASE1, dict(tol_lo=delta, tol_hi=delta))
        st, obj, _ = simplex.solve_dense(lp, ops)
        assert st == "optimal"
        objs.append(obj)
    assert objs[0] >= objs[1] - 1e-12 >= objs[2] - 2e-12


def test_planted_sign_error_is_caught(monkeypatch):
    """A sign slip in the detector coordinate (y sin -> -y sin) breaks the disc pin."""
    import oracle.operators as O
    orig = O.detector_coordinate

    def flipped(x, y, c, s, off, precision="f64"):
        return orig(x, -y, c, s, off, precision)

    monkeypatch.setattr(O, "detector_coordinate", flipped)
    n, r = 64, 14
    cx, cy = 0.07 * n, -0.05 * n
    c = np.arange(n) - (n - 1) / 2
    Y, X = np.meshgrid(c, c, indexing="ij")
    f = ((X - cx) ** 2 + (Y - cy) ** 2 <= r * r).astype(float)
    th = 1.0
    geo = Geometry(n, n, 1, np.array([th]), 93)
    p = O.Operators(geo).project_raw(f[:, :, None])[0, :, 0]
    s = np.arange(93) - 46.0
    s0 = cx * math.cos(th) + cy * math.sin(th)
    ana = 2 * np.sqrt(np.maximum(r * r - (s - s0) ** 2, 0))
    assert np.linalg.norm(p - ana) / np.linalg.norm(ana) > 0.05


def _best_certificate(lp, ops):
    """Largest obj - B * kappa over candidates of the bound-based certificate,
    as an LP for HiGHS in (lam_up on its rows, lam_lo on gel, t) with
    sum lam <= 1: t >= kappa is enforced by A(lam_up - lam_lo) + t b >= 0 on
    every active ray.  lam_up lives on band rows (Case 2, bound 1) or gel
    rows (Case 1, bound f~_U).  Returns the value and the maximiser as
    full-length dual vectors."""
    act = np.flatnonzero(lp.active)
    gel = np.flatnonzero(lp.gel)
    up = np.flatnonzero(lp.band) if lp.case == CASE2 else gel
    U = np.ones(up.size) if lp.case == CASE2 else lp.upper[gel]
    b, B, _ = pdhg.certificate_data(lp, ops)
    Au = ops.PT[up][:, act].T.toarray()
    Ag = ops.PT[gel][:, act].T.toarray()
    nu, ng = up.size, gel.size
    G = np.hstack([-Au, Ag, -b[act][:, None]])
    G = np.vstack([G, np.concatenate([np.ones(nu + ng), [0.0]])[None, :]])
    h = np.concatenate([np.zeros(act.size), [1.0]])
    c = np.concatenate([U, -lp.lower[gel], [B]])      # minimise -(obj - B t)
    res = linprog(c, A_ub=G, b_ub=h, bounds=[(0, None)] * (nu + ng + 1), method="highs")
    assert res.status == 0
    lu = np.zeros(lp.labels.size)
    ll = np.zeros(lp.labels.size)
    lu[up] = res.x[:nu]
    ll[gel] = res.x[nu:nu + ng]
    return -res.fun, lu, ll


def test_bound_certificate_is_sound_and_complete_on_tiny_lps():
    """Farkas with the ray bound: on a feasible LP (simplex optimum) no
    candidate gives obj > B kappa, so the test cannot fire; on an infeasible
    one (simplex: infeasible) the best candidate does and the oracle's test
    accepts it."""
    lp, ops = _tiny(CASE2, dict(inhibit_ratio=0.6))
    assert simplex.solve_dense(lp, ops)[0] == "optimal"
    val, lu, ll = _best_certificate(lp, ops)
    assert val <= 1e-9
    assert not pdhg.certificate(lp, ops, lu, ll, *pdhg.certificate_data(lp, ops))
    lp, ops = _tiny(CASE2, dict(inhibit_ratio=0.3))
    assert simplex.solve_dense(lp, ops)[0] == "infeasible"
    val, lu, ll = _best_certificate(lp, ops)
    assert val > 1e-3
    assert pdhg.certificate(lp, ops, lu, ll, *pdhg.certificate_data(lp, ops))


@pytest.mark.parametrize("delta", [0.0, 0.05])
def test_bound_certificate_cannot_fire_on_feasible_case1(delta):
    """Case 1 (lam_up on gel rows, bound f~_U): on feasible LPs, down to the
    equality case delta = 0, the best candidate HiGHS finds has
    obj - B kappa <= 0 and the oracle's test rejects it."""
    lp, ops = _tiny(CASE1, dict(tol_lo=delta, tol_hi=delta))
    assert simplex.solve_dense(lp, ops)[0] == "optimal"
    val, lu, ll = _best_certificate(lp, ops)
    assert val <= 1e-9
    assert not pdhg.certificate(lp, ops, lu, ll, *pdhg.certificate_data(lp, ops))


def test_bound_certificate_detects_blurred_inhibition(monkeypatch):
    """A blurred, attenuated 16^3 Case-2 part at r = 0.8: the blur makes the
    in-part / out-of-part contrast unreachable; the bound-based certificate
    proves it within 1024 iterations, where the l_inf ray test alone does not."""
    from synthetic.targets import csg_3d
    n = 16
    tgt = csg_3d(n, vial_radius=n * 0.47, band_width=2, seed=2, feature=(3.0, 6.0))
    geo = Geometry(n, n, n, uniform_angles(24), n, vial_radius=n * 0.47, mu=0.08,
                   psf_sigma=(1.5, 1.5, 2.5))
    lp, ops = build_lp(geo, tgt, CaseParams(case=CASE2, inhibit_ratio=0.8, band_width=2))
    res = pdhg.solve(lp, ops, kkt_tol=1e-4, max_iter=1024)
    assert res["status"] == pdhg.PRIMAL_INFEASIBLE
    monkeypatch.setattr(pdhg, "certificate", lambda *a: False)
    res = pdhg.solve(lp, ops, kkt_tol=1e-4, max_iter=1024)
    assert res["status"] == pdhg.ITER_LIMIT


def test_disc64_golden_matches_highs():
    """The stored Case-1 optimum of the 64x64 / 96-angle / 91-bin workload
    (tests/golden/disc64_case1.json, written by the oracle's PDHG) against
    scipy's HiGHS on the same LP (Eqs. 32-37, delta = 0.05); its interior-point
    method with crossover finishes in seconds where the simplex takes minutes."""
    import json
    import os
    from synthetic.targets import workload
    with open(os.path.join(os.path.dirname(__file__), "golden", "disc64_case1.json")) as f:
        gold = json.load(f)
    wl = workload("disc64")
    lp, ops = build_lp(Geometry(64, 64, 1, wl.angles, 91), wl.target,
                       CaseParams(case=CASE1, tol_lo=0.05, tol_hi=0.05, band_width=10))
    ref = _highs(lp, ops, method="highs-ipm")
    assert ref.status == 0
    assert abs(gold["objective"] - ref.fun) <= 1e-7 * abs(ref.fun)


def _slice_stack(nz, bad_z, ratio=0.62):
    """Case 2 on a stack of 12x12 slices (10 views, 17 bins): every slice holds
    a disc pattern feasible at this ratio except slice bad_z, whose disc needs
    more contrast than the ratio allows (thresholds found by HiGHS below)."""
    n, na, nd = 12, 10, 17
    feas = [discs_2d(n, n_discs=1, r_range=(2.5, 3.5), container_radius=4.5, seed=3),
            discs_2d(n, n_discs=3, r_range=(1.0, 1.6), container_radius=4.5, seed=3),
            discs_2d(n, n_discs=1, r_range=(2.5, 3.5), container_radius=4.5, seed=5)]
    bad = discs_2d(n, n_discs=1, r_range=(2.5, 3.5), container_radius=4.5, seed=1)
    sl = [feas[i % 3] for i in range(nz)]
    if bad_z is not None:
        sl[bad_z] = bad
    tgt = np.concatenate(sl, axis=2)
    return build_lp(Geometry(n, n, nz, uniform_angles(na), nd), tgt,
                    CaseParams(case=CASE2, inhibit_ratio=ratio, band_width=2))


def _slice_rows_rays(lp, ops, z):
    """2-D indices (into the per-slice matrix ops.PT) of slice z's band rows,
    gel rows and active rays, and their flat 3-D indices."""
    nz = ops.geo.nz
    vz = np.arange(lp.labels.size) % nz == z
    band3, gel3 = np.flatnonzero(lp.band & vz), np.flatnonzero(lp.gel & vz)
    act3 = np.flatnonzero(lp.active & (np.arange(lp.active.size) % nz == z))
    return band3 // nz, gel3 // nz, act3 // nz, band3, gel3, act3


def _slice_feasible(lp, ops, z):
    """HiGHS on the rows and rays of slice z alone (the operator is P_2D on
    every slice, block diagonal over z without a z-extent PSF)."""
    band, gel, act, _, gel3, _ = _slice_rows_rays(lp, ops, z)
    M = ops.PT[:, act]
    G = sp.vstack([M[band], -M[gel]]).tocsr()
    h = np.concatenate([np.ones(band.size), -lp.lower[gel3]])
    r = linprog(np.zeros(act.size), A_ub=G, b_ub=h, bounds=[(0, None)] * act.size, method="highs")
    return r.status == 0


def _slice_best_certificate(lp, ops, z):
    """_best_certificate restricted to slice z: the largest obj_z - B_z kappa_z
    and its maximiser embedded in full-length dual vectors."""
    up, gel, act, up3, gel3, act3 = _slice_rows_rays(lp, ops, z)
    b, _, B_z = pdhg.certificate_data(lp, ops)
    Au = ops.PT[up][:, act].T.toarray()
    Ag = ops.PT[gel][:, act].T.toarray()
    nu, ng = up.size, gel.size
    G = np.hstack([-Au, Ag, -b[act3][:, None]])
    G = np.vstack([G, np.concatenate([np.ones(nu + ng), [0.0]])[None, :]])
    h = np.concatenate([np.zeros(act.size), [1.0]])
    c = np.concatenate([np.ones(nu), -lp.lower[gel3], [B_z[z]]])
    res = linprog(c, A_ub=G, b_ub=h, bounds=[(0, None)] * (nu + ng + 1), method="highs")
    assert res.status == 0
    lu = np.zeros(lp.labels.size)
    ll = np.zeros(lp.labels.size)
    lu[up3] = res.x[:nu]
    ll[gel3] = res.x[nu:nu + ng]
    return -res.fun, lu, ll


def test_per_slice_certificate_is_sound_and_names_the_slice():
    """Without a z-extent PSF the LP is feasible iff every slice is (HiGHS per
    slice).  The best per-slice candidate of each feasible slice cannot pass the
    slice test; the infeasible slice's passes it.  Add a small uniform lam_lo
    on the gel rows of every other slice (the residue an iteration leaves on
    feasible slices): the slice test still accepts, the whole-volume test,
    whose kappa is a maximum over all slices and whose B sums them, does not."""
    nz, bad_z = 8, 4
    lp, ops = _slice_stack(nz, bad_z)
    assert pdhg.slices_decoupled(ops)
    feasible = [_slice_feasible(lp, ops, z) for z in range(nz)]
    assert feasible == [z != bad_z for z in range(nz)]
    data = pdhg.certificate_data(lp, ops)
    for z in range(nz):
        val, lu, ll = _slice_best_certificate(lp, ops, z)
        if z == bad_z:
            assert val > 1e-3
            assert pdhg.certificate(lp, ops, lu, ll, *data)
            other = lp.gel & (np.arange(lp.labels.size) % nz != z)
            ll2 = ll + 1e-4 * other
            assert pdhg.certificate(lp, ops, lu, ll2, *data)
            assert not pdhg.certificate(lp, ops, lu, ll2, *data, per_slice=False)
        else:
            assert val <= 1e-9
            assert not pdhg.certificate(lp, ops, lu, ll, *data)


def test_per_slice_certificate_ends_the_solve_sooner(monkeypatch):
    """The oracle PDHG on the 16-slice stack with one infeasible slice: with the
    l_inf ray test switched off, the slice test proves infeasibility within
    5120 iterations; the whole-volume test alone needs more."""
    lp, ops = _slice_stack(16, 8)
    monkeypatch.setattr(pdhg, "_farkas", lambda *a, **k: False)
    res = pdhg.solve(lp, ops, kkt_tol=1e-7, max_iter=5120)
    assert res["status"] == pdhg.PRIMAL_INFEASIBLE
    whole = pdhg.certificate
    monkeypatch.setattr(pdhg, "certificate", lambda *a, **k: whole(*a, per_slice=False))
    res = pdhg.solve(lp, ops, kkt_tol=1e-7, max_iter=5120)
    assert res["status"] == pdhg.ITER_LIMIT


def test_separation_lp_settles_case2_feasibility():
    """The separation LP minimises the band-to-gel dose ratio: in the general
    form with w1 = 1, w2 = 0, or as Case 1 with tol_lo = 0 and tol_hi = 10 (the
    gel upper rows are slack at the optimum here), both optima equal (HiGHS).
    Case 2 at ratio r is feasible iff u~* <= r: above it the separation LP's
    optimal dual (either form) passes the bound-based Farkas test of the
    Case-2 LP; below it the separation point over r satisfies every Case-2 row
    (Eqs. 40-45)."""
    r = 0.62
    for bad in (8, None):
        lp2, ops2 = _slice_stack(16, bad, ratio=r)
        tgt = lp2.f_T.reshape(12, 12, 16)
        lp0, ops0 = build_lp(ops2.geo, tgt, CaseParams(case=GENERAL, w1=1.0, w2=0.0, band_width=2))
        lp1, ops1 = build_lp(ops2.geo, tgt, CaseParams(case=CASE1, tol_lo=0.0, tol_hi=10.0, band_width=2))
        ref0 = _highs(lp0, ops0, method="highs-ipm")
        ref1 = _highs(lp1, ops1, method="highs-ipm")
        assert abs(ref0.fun - ref1.fun) <= 1e-7 * ref0.fun
        for lp, ops, ref in ((lp0, ops0, ref0), (lp1, ops1, ref1)):
            res = pdhg.solve(lp, ops, kkt_tol=1e-6, max_iter=100000)
            assert res["status"] == pdhg.OPTIMAL and abs(res["obj"] - ref.fun) <= 1e-5 * ref.fun
            cert = pdhg.certificate(lp2, ops2, res["lam_up"], res["lam_lo"], *pdhg.certificate_data(lp2, ops2))
            if bad is not None:
                assert ref.fun > r and cert
            else:
                assert ref.fun < r and not cert
                y = res["y"] / r
                d = ops2.AT(y.reshape(ops2.geo.sino_shape)).ravel()
                assert np.all(d[lp2.band] <= 1.0 + 1e-5) and np.all(d[lp2.gel] >= lp2.lower[lp2.gel] * (1 - 1e-5))


def test_empty_band_reading():
    """band_width 0 without a PSF: the band of Sec. 2.2 (supp(K f_T) minus the
    gel, K = I) is empty.  With u~ free (Eqs. 9-24) and in no row, Case 1 and
    the general form are unbounded - the dense simplex says so - and the
    oracle refuses to build them; Case 2 has no u~ and stays a proper LP, its
    PDHG optimum equal to the simplex's."""
    tgt = discs_2d(10, n_discs=1, r_range=(2.0, 3.0), container_radius=4.0, seed=3)
    geo = Geometry(10, 10, 1, uniform_angles(8), 15)
    for case, extra in ((GENERAL, {}), (CASE1, dict(tol_lo=0.1, tol_hi=0.1))):
        with pytest.raises(ValueError, match="empty band"):
            build_lp(geo, tgt, CaseParams(case=case, band_width=0, **extra))
    # the same LP written out without the refusal: unbounded for the simplex
    lp, ops = build_lp(geo, tgt, CaseParams(case=CASE1, tol_lo=0.1, tol_hi=0.1, band_width=1))
    lp.labels = np.where(lp.labels == BAND, EXT, lp.labels).astype(np.uint8)   # band rows removed
    assert not lp.band.any()
    assert simplex.solve_dense(lp, ops)[0] == "unbounded"
    lp2, ops2 = build_lp(geo, tgt, CaseParams(case=CASE2, inhibit_ratio=0.6, band_width=0))
    assert not lp2.band.any()
    st, obj, _ = simplex.solve_dense(lp2, ops2)
    res = pdhg.solve(lp2, ops2, kkt_tol=1e-9, max_iter=100000)
    assert st == "optimal" and res["status"] == pdhg.OPTIMAL
    assert abs(res["obj"] - obj) <= 1e-7 * abs(obj)
