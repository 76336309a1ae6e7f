"""Pins for the oracle's scale-invariant metrics (CPU only).

`oracle.lp.metrics` is checked against values fixed by hand arithmetic on a
five-voxel dose field (DTVR of Eq. 6/8, DSR in both of its printed forms,
Eq. 7 and Eq. 8, PSR_f of Eq. 46, the post-scaling factor of Eq. 27 and the
recovered Charnes-Cooper scale), and against the identities the LP optimum
must satisfy (Sec. 2.6.2, Sec. 2.7): the fractional objective of the
optimal dose equals the LP objective, which ties DSR and PSR_f of a
binary-target Case-1 optimum to u~*.
"""
import numpy as np
import pytest

from oracle import simplex
from oracle.lp import BAND, CASE1, CASE2, EXT, GEL, GENERAL, CaseParams, LPData, build_lp, metrics
from oracle.operators import Geometry
from synthetic.targets import discs_2d, uniform_angles


def _five_voxel_lp(case, f_crit):
    """Labels gel, gel, band, band, ext; f_T = 2, 4 on the gel voxels."""
    lab = np.array([GEL, GEL, BAND, BAND, EXT], np.uint8)
    f_T = np.array([2.0, 4.0, 0.0, 0.0, 0.0])
    ft = np.where(lab == GEL, f_T / f_crit, 0.0)
    return LPData(case=case, labels=lab, ft=ft, lower=ft.copy(), upper=np.zeros(5),
                  active=np.ones(1, bool), f_crit=f_crit, f_T=f_T, c_u=1.0, c_v=1.0)


DOSE = np.array([3.0, 10.0, 1.5, 0.5, 7.0])


def test_metrics_of_a_hand_computed_dose_field():
    """General form, f_crit = min_gel f_T = 2, so f~_T = (1, 2) on gel.
    d / f~_T = (3, 5): DTVR = 5/3.  DSR (Eq. 8) = max_band d / min_gel(d / f~_T)
    = 1.5 / 3.  PSR_f (Eq. 46) = min_gel d / max_band d = 3 / 1.5 (an inverted
    ratio, band over gel, would give 0.5; counting the exterior voxel's 7 as
    band would give DSR 7/3 and PSR_f 3/7).  alpha* (Eq. 27, unit weights)
    = <d, f_T>_gel / <d, d>_gel = (3*2 + 10*4) / (9 + 100).  s = min_gel d / f~_L
    = min(3/1, 10/2) = 3."""
    m = metrics(_five_voxel_lp(GENERAL, 2.0), DOSE)
    assert m["dtvr_f"] == pytest.approx(5.0 / 3.0, rel=1e-15)
    assert m["dsr"] == pytest.approx(0.5, rel=1e-15)
    assert m["psr_f"] == pytest.approx(2.0, rel=1e-15)
    assert m["alpha"] == pytest.approx(46.0 / 109.0, rel=1e-15)
    assert m["s"] == pytest.approx(3.0, rel=1e-15)
    assert m["band_max"] == 1.5


def test_dsr_printed_forms_agree():
    """Eq. 7 divides the band maximum by f_crit and the gel doses by f_T; Eq. 8
    uses f~_T = f_T / f_crit.  With f_crit = 1.6 (Case 2 at r = 0.8 of
    min f_T = 2): Eq. 7 = (1.5 / 1.6) / min(3/2, 10/4) = 0.625.  DTVR and PSR_f
    do not depend on f_crit."""
    m = metrics(_five_voxel_lp(CASE2, 1.6), DOSE)
    assert m["dsr"] == pytest.approx((1.5 / 1.6) / 1.5, rel=1e-15)
    assert m["dsr"] == pytest.approx(0.625, rel=1e-15)
    assert m["dtvr_f"] == pytest.approx(5.0 / 3.0, rel=1e-15)
    assert m["psr_f"] == pytest.approx(2.0, rel=1e-15)


def _tiny(case, extra, seed=3):
    tgt = discs_2d(10, n_discs=1, r_range=(2.0, 3.0), container_radius=4.0, seed=seed)
    geo = Geometry(10, 10, 1, uniform_angles(8), 15)
    return build_lp(geo, tgt, CaseParams(case=case, band_width=2, **extra))


@pytest.mark.parametrize("delta", [0.05, 0.1, 0.2])
def test_case1_optimum_fixes_dsr_and_psr(delta):
    """Case 1 on a binary target (Sec. 2.7.1): f_crit = (1 - delta) min f_T, so
    f~_T = 1 / (1 - delta) and the lower rows read d >= 1 on gel.  At the LP
    optimum the lower bound is attained (otherwise scaling y down lowers u~),
    so min_gel d = 1 and max_band d = u~*: DSR = u~* / (1 - delta) and
    PSR_f = 1 / u~*.  The simplex optimum's dose is used, so the pin does not
    rest on the PDHG."""
    lp, ops = _tiny(CASE1, dict(tol_lo=delta, tol_hi=delta))
    st, obj, y = simplex.solve_dense(lp, ops)
    assert st == "optimal"
    d = ops.AT(y.reshape(ops.geo.sino_shape)).ravel()
    m = metrics(lp, d)
    assert m["dsr"] == pytest.approx(obj / (1.0 - delta), rel=1e-9)
    assert m["psr_f"] == pytest.approx(1.0 / obj, rel=1e-9)
    assert m["s"] == pytest.approx(1.0, rel=1e-9)
