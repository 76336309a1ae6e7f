"""GPU response-domain front and back end against the oracle (Sec. 2.1, Eqs. 4-5,
28, 46; Case 1 with response tolerances, Sec. 2.7.1).

The map is computed in FP64 from float32 inputs on both sides, so the GPU's
float32 outputs agree with the oracle to output rounding.  The explicit-bound
Case 1 gets the same float32 bounds on both sides, so FP64 iterates agree to
rounding while no restart decision flips.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle import pdhg
from oracle.lp import CaseParams, build_lp
from oracle.operators import Geometry
from oracle.response import Richards as ORichards
from oracle.response import alpha_m, dose_bounds, phi_m, response, response_inverse, response_metrics
from synthetic.targets import graded_discs_2d, uniform_angles

MP = (0.0, 1.0, 8.0, 0.7, 0.5)       # alpha, k, beta, gamma, f0


@pytest.fixture(scope="module")
def sipo():
    import paper_2604_08997_gb300 as s
    s.build()
    return s


def test_response_map_matches_the_oracle(sipo):
    rng = np.random.default_rng(11)
    M = sipo.Richards(*MP)
    OM = ORichards(*MP)
    m = rng.uniform(-0.1, 0.999, 100_003).astype(np.float32)
    m[:3] = (0.0, -0.0, 1e-7)
    got = sipo.response_to_dose(M, m).cpu().numpy()
    ref = response_inverse(OM, m.astype(np.float64))
    np.testing.assert_allclose(got, ref, rtol=1e-6, atol=1e-7)
    assert np.all(got[m <= 0] == 0)
    got2 = sipo.response_to_dose(M, m, 0.5).cpu().numpy()
    np.testing.assert_allclose(got2, response_inverse(OM, 0.5 * m.astype(np.float64)), rtol=1e-6, atol=1e-7)
    f = rng.uniform(-1.0, 2.0, 50_001).astype(np.float32)
    np.testing.assert_allclose(sipo.dose_to_response(M, f).cpu().numpy(), response(OM, f.astype(np.float64)),
                               rtol=1e-6, atol=1e-7)
    with pytest.raises(sipo.SipoError):
        sipo.response_to_dose(M, np.array([0.5, 1.0], np.float32))


def _response_target():
    n, na, nd = 10, 8, 15
    m_T = graded_discs_2d(n, levels=(0.7, 0.6, 0.5), r_range=(1.5, 3.0), container_radius=4.0, seed=4)
    ang = uniform_angles(na)
    return m_T, ang, Geometry(n, n, 1, ang, nd), dict(nx=n, ny=n, nz=1, angles=ang, n_det=nd)


def test_explicit_bounds_track_the_oracle(sipo):
    """sipo_create_bounded with response-domain bounds (float32 on both sides):
    FP64 iterates, objectives and restart counts match the oracle PDHG on the
    same explicit-bound LP for 320 iterations."""
    m_T, ang, geom, geo = _response_target()
    f_T, f_L, f_U = (a.astype(np.float32) for a in dose_bounds(ORichards(*MP), m_T, 0.05, 0.05))
    lp, ops = build_lp(geom, f_T, CaseParams(case=1, band_width=2, f_lower=f_L.astype(np.float64),
                                             f_upper=f_U.astype(np.float64)))
    ref = pdhg.solve(lp, ops, kkt_tol=0.0, max_iter=320)
    ctx = sipo.sipo_create_bounded(geo, f_T, f_L, f_U, dict(band_width=2),
                                   dict(storage=sipo.SIPO_F64, kkt_tol=0.0, max_iter=320))
    res = sipo.sipo_solve(ctx)
    assert res["iters"] == 320 and res["restarts"] == ref["restarts"]
    assert abs(res["f_crit"] - lp.f_crit) <= 1e-15 * lp.f_crit
    for key in ("pobj", "dobj", "rel_primal", "rel_dual"):
        a, b = res[key], ref["info"][key]
        assert abs(a - b) <= 1e-7 * max(abs(b), 1e-3), (key, a, b)
    with pytest.raises(sipo.SipoError):          # an upper bound below the lower one
        sipo.sipo_create_bounded(geo, f_T, f_L, (0.5 * f_L).astype(np.float32), dict(band_width=2),
                                 dict(storage=sipo.SIPO_F64))


def test_response_case1_solve_and_metrics_match_the_oracle(sipo):
    """response_case1 (front end on the device) solved in FP64 and FP32 reaches
    the oracle optimum; sipo_response_metrics post-scales in the response
    domain (Eq. 28) to the oracle's minimiser and reports PSR_m / DTVR_m as the
    oracle does on the GPU's own dose."""
    m_T, ang, geom, geo = _response_target()
    OM = ORichards(*MP)
    f_T, f_L, f_U = (a.astype(np.float32) for a in dose_bounds(OM, m_T, 0.05, 0.05))
    lp, ops = build_lp(geom, f_T, CaseParams(case=1, band_width=2, f_lower=f_L.astype(np.float64),
                                             f_upper=f_U.astype(np.float64)))
    ref = pdhg.solve(lp, ops, kkt_tol=1e-10, max_iter=100000)
    assert ref["status"] == pdhg.OPTIMAL
    M = sipo.Richards(*MP)
    for storage, tol, rel in ((sipo.SIPO_F64, 1e-10, 1e-7), (sipo.SIPO_F32, 1e-5, 1e-4)):
        ctx = sipo.response_case1(geo, m_T, M, 0.05, 0.05, band_width=2,
                                  tolerances=dict(storage=storage, kkt_tol=tol, max_iter=100000))
        y = np.empty(len(ang) * 15, np.float64 if storage == sipo.SIPO_F64 else np.float32)
        res = sipo.sipo_solve(ctx, y)
        assert res["status"] == sipo.SIPO_OPTIMAL, res
        assert abs(res["pobj"] - ref["obj"]) <= rel * ref["obj"]
        if storage != sipo.SIPO_F64:
            continue
        d = ops.AT(y.astype(np.float64).reshape(geom.sino_shape)).ravel()
        got = sipo.response_metrics(ctx, M, m_T)
        a_ref = alpha_m(OM, d, m_T, lp.gel, res["alpha"])
        assert abs(got["alpha"] - a_ref) <= 1e-4 * a_ref
        assert got["phi"] <= phi_m(OM, a_ref, d, m_T, lp.gel) * (1 + 1e-6) + 1e-15
        want = response_metrics(OM, lp, d, m_T, got["alpha"])
        for key in ("phi", "psr_m", "dtvr_m", "ratio_min", "ratio_max", "m_band_max", "m_gel_min"):
            assert abs(got[key] - want[key]) <= 1e-9 * abs(want[key]), (key, got[key], want[key])
        fixed = sipo.response_metrics(ctx, M, m_T, alpha=0.6)
        want = response_metrics(OM, lp, d, m_T, 0.6)
        assert fixed["alpha"] == 0.6 and abs(fixed["psr_m"] - want["psr_m"]) <= 1e-9 * want["psr_m"]


def test_response_case2_threshold_is_the_response_threshold(sipo):
    """Case 2 with the inhibition threshold given as a response: f_crit = M^-1(m_crit)."""
    m_T, ang, geom, geo = _response_target()
    M = sipo.Richards(*MP)
    ctx = sipo.response_case2(geo, m_T, M, 0.33, band_width=2,
                              tolerances=dict(storage=sipo.SIPO_F64, kkt_tol=1e-6, max_iter=2000))
    res = sipo.sipo_solve(ctx)
    want = float(response_inverse(ORichards(*MP), np.array([0.33]))[0])
    assert abs(res["f_crit"] - want) <= 1e-6 * want


def test_response_inhibit_ratio_on_the_device(sipo):
    """sipo_response_inhibit_ratio: the part's smallest prescribed response and
    r = M^-1(m_crit) / M^-1(min m_T) against the oracle's inverse in FP64; a
    threshold outside (alpha, k) and a target without a part are refused."""
    from paper_2604_08997_gb300._abi import sipo_response_inhibit_ratio
    m_T, *_ = _response_target()
    m = torch.from_numpy(np.ascontiguousarray(m_T)).cuda()
    r, gmin = sipo_response_inhibit_ratio(MP, m, 0.33)
    OM = ORichards(*MP)
    assert gmin == pytest.approx(float(m_T[m_T > 0].min()), rel=0, abs=0)
    want = float(response_inverse(OM, np.array([0.33]))[0] / response_inverse(OM, np.array([gmin]))[0])
    assert r == pytest.approx(want, rel=1e-12)
    with pytest.raises(sipo.SipoError):
        sipo_response_inhibit_ratio(MP, m, 1.5)
    with pytest.raises(sipo.SipoError):
        sipo_response_inhibit_ratio(MP, torch.zeros(16, device="cuda"), 0.33)
