"""Pins for the oracle's material response (Sec. 2.1, Eqs. 4-5, 28, 46) and for
Case 1 with explicit per-voxel dose bounds (Sec. 2.7.1 response tolerances).

Richards' curve is pinned to the textbook logistic (gamma = 1, scipy's
expit), its closed-form inverse to a bracketing root finder, the response
post-scaling to a brute-force scan, and PSR_m to its monotone shortcut.  The
explicit-bound LP is pinned to the proportional Case 1 it generalises and to
HiGHS on the LP written in dose units from the definitions.
"""
import numpy as np
import pytest
import scipy.sparse as sp
from scipy.optimize import brentq, linprog
from scipy.special import expit

from oracle import pdhg
from oracle.lp import BAND, CASE1, GEL, CaseParams, build_lp
from oracle.operators import Geometry
from oracle.response import (Richards, alpha_m, dose_bounds, phi_m, response, response_inverse,
                             response_metrics)
from synthetic.targets import graded_discs_2d, uniform_angles

M = Richards(alpha=0.0, k=1.0, beta=8.0, gamma=0.7, f0=0.5)


def test_richards_with_unit_shape_is_the_logistic():
    f = np.linspace(-1.0, 2.0, 301)
    p = Richards(0.1, 0.9, 6.0, 1.0, 0.4)
    np.testing.assert_allclose(response(p, f), 0.1 + 0.8 * expit(6.0 * (f - 0.4)), rtol=0, atol=1e-15)


def test_richards_inverse_matches_a_root_finder():
    rng = np.random.default_rng(3)
    for p in (M, Richards(0.05, 0.95, 3.0, 2.5, 1.0)):
        ms = rng.uniform(p.alpha + 1e-3, p.k - 1e-3, 50)
        got = response_inverse(p, ms)
        for m, f in zip(ms, got):
            ref = brentq(lambda x: float(response(p, x)) - m, -50.0, 50.0, xtol=1e-14, rtol=1e-15)
            assert abs(f - ref) <= 1e-9 * max(1.0, abs(ref))
        np.testing.assert_allclose(response(p, got), ms, rtol=1e-12)


def test_richards_limits_and_range():
    assert abs(float(response(M, -1e3)) - M.alpha) < 1e-15
    assert abs(float(response(M, 1e3)) - M.k) < 1e-15
    f = np.linspace(-2, 3, 500)
    assert np.all(np.diff(response(M, f)) >= 0)
    assert np.array_equal(response_inverse(M, np.array([0.0, -0.2])), np.zeros(2))
    with pytest.raises(ValueError):
        response_inverse(M, np.array([0.5, 1.0]))


def _response_lp(case_extra=None):
    m_T = graded_discs_2d(10, levels=(0.7, 0.6, 0.5), r_range=(1.5, 3.0), container_radius=4.0, seed=4)
    f_T, f_L, f_U = dose_bounds(M, m_T, 0.05, 0.05)
    geo = Geometry(10, 10, 1, uniform_angles(8), 15)
    lp, ops = build_lp(geo, f_T, CaseParams(case=CASE1, band_width=2, f_lower=f_L, f_upper=f_U))
    return m_T, f_T, f_L, f_U, geo, lp, ops


def test_response_bounds_are_not_proportional_to_the_target():
    """Through M^-1 the dose interval of each level differs in relative width
    (Sec. 2.7.1), which is why Case 1 takes explicit per-voxel bounds."""
    m_T, f_T, f_L, f_U, _, lp, _ = _response_lp()
    gel = m_T.ravel() > 0
    ratio = f_U.ravel()[gel] / f_L.ravel()[gel]
    assert ratio.max() - ratio.min() > 1e-3
    assert np.all(f_L.ravel()[gel] < f_T.ravel()[gel]) and np.all(f_T.ravel()[gel] < f_U.ravel()[gel])
    assert abs(lp.f_crit - f_L.ravel()[gel].min()) == 0.0
    np.testing.assert_array_equal(lp.upper[lp.gel], f_U.ravel()[lp.gel] / lp.f_crit)


def test_explicit_proportional_bounds_reproduce_case1():
    """f_L = (1 - d) f_T, f_U = (1 + d) f_T passed explicitly give the proportional
    Case-1 LP: same data up to rounding, same PDHG iterates."""
    f_T = graded_discs_2d(10, levels=(1.0, 0.85, 0.7), r_range=(1.5, 3.0), container_radius=4.0, seed=4)
    geo = Geometry(10, 10, 1, uniform_angles(8), 15)
    f64 = f_T.astype(np.float64)
    lp1, ops = build_lp(geo, f_T, CaseParams(case=CASE1, band_width=2, tol_lo=0.1, tol_hi=0.1))
    lp2, _ = build_lp(geo, f_T, CaseParams(case=CASE1, band_width=2, f_lower=0.9 * f64, f_upper=1.1 * f64))
    np.testing.assert_allclose(lp2.lower, lp1.lower, rtol=1e-15)
    np.testing.assert_allclose(lp2.upper, lp1.upper, rtol=1e-15)
    r1 = pdhg.solve(lp1, ops, kkt_tol=0.0, max_iter=256)
    r2 = pdhg.solve(lp2, ops, kkt_tol=0.0, max_iter=256)
    assert r1["restarts"] == r2["restarts"]
    assert abs(r1["obj"] - r2["obj"]) <= 1e-12 * abs(r1["obj"])


def _dose_unit_case1(f_L, f_U, ops, lp):
    """Case 1 in dose units from its definition: min u s.t. f_L <= f <= f_U on gel,
    f <= u min_gel f_L on band, f = P^T y over active rays, y >= 0."""
    act = np.flatnonzero(lp.active)
    Mx = ops.PT[:, act]
    gel, band = np.flatnonzero(lp.labels == GEL), np.flatnonzero(lp.labels == BAND)
    lo, hi = f_L.ravel()[gel].astype(np.float64), f_U.ravel()[gel].astype(np.float64)
    fc = lo.min()
    nb, ng = band.size, gel.size
    ucol = sp.csr_matrix((-np.full(nb, fc), (np.arange(nb), np.zeros(nb, int))), shape=(nb, 1))
    G = sp.vstack([sp.hstack([Mx[band], ucol]), sp.hstack([Mx[gel], sp.csr_matrix((ng, 1))]),
                   sp.hstack([-Mx[gel], sp.csr_matrix((ng, 1))])]).tocsr()
    h = np.concatenate([np.zeros(nb), hi, -lo])
    c = np.zeros(act.size + 1)
    c[-1] = 1.0
    return linprog(c, A_ub=G, b_ub=h, bounds=[(0, None)] * (act.size + 1), method="highs")


def test_response_case1_matches_dose_unit_lp():
    m_T, f_T, f_L, f_U, geo, lp, ops = _response_lp()
    ref = _dose_unit_case1(f_L, f_U, ops, lp)
    assert ref.status == 0
    res = pdhg.solve(lp, ops, kkt_tol=1e-10, max_iter=100000)
    assert res["status"] == pdhg.OPTIMAL
    assert abs(res["obj"] - ref.fun) <= 1e-8 * ref.fun


def test_response_post_scaling_and_metrics():
    """alpha_m minimises Phi_m (Eq. 28) to the resolution of a dense scan; the
    metrics follow their definitions (PSR_m through the monotone M equals
    M(alpha min_gel d) / M(alpha max_band d), Eq. 46)."""
    m_T, f_T, f_L, f_U, geo, lp, ops = _response_lp()
    res = pdhg.solve(lp, ops, kkt_tol=1e-8, max_iter=100000)
    d = res["d"]
    centre = res["metrics"]["alpha"]
    a = alpha_m(M, d, m_T, lp.gel, centre)
    scan = centre * np.linspace(0.05, 4.0, 20001)
    best = min(phi_m(M, x, d, m_T, lp.gel) for x in scan)
    assert phi_m(M, a, d, m_T, lp.gel) <= best * (1 + 1e-9) + 1e-15
    met = response_metrics(M, lp, d, m_T, a)
    dg, db = d[lp.gel], d[lp.band]
    assert abs(met["psr_m"] - float(response(M, a * dg.min()) / response(M, a * db.max()))) <= 1e-12
    assert met["dtvr_m"] >= 1.0 and met["ratio_min"] <= 1.0 + 1e-3
