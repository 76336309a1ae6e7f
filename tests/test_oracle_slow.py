"""The measured workload's Case 2 at r = 0.8 settled on the CPU (slow: about 8
minutes; runs with SIPO_SLOW=1).

The 256^3 x 360-view part (seed 2) at inhibition ratio 0.8 asks for band dose
<= 1 and gel dose >= 1.25 (normalised).  The forward model is slice-separable
(Sec. 2.3), so one infeasible z-slice makes the whole LP infeasible.  On slice
138, with the labels of the 3-D part, the oracle solves the separation LP
(Case 1 with tol_lo = 0, tol_hi = 10: least band maximum with gel dose at
least its target) in FP64 and tests its dual point as a Farkas ray of the
Case-2 rows of that slice with the bound-based test (Secs. 2.7.1-2.7.2).  A
passing ray proves the Case-2 LP infeasible by itself, whatever the accuracy
of the iterate; the separation optimum, about 0.814 > 0.8, says the same in
ratio terms.
"""
import os

import numpy as np
import pytest

from oracle import pdhg
from oracle.lp import CaseParams, build_lp, partition
from oracle.operators import Geometry
from synthetic.targets import workload

pytestmark = [pytest.mark.slow,
              pytest.mark.skipif(not os.environ.get("SIPO_SLOW"), reason="slow: set SIPO_SLOW=1")]


def test_csg256_ratio_08_is_infeasible_on_slice_138():
    z, r = 138, 0.8
    wl = workload("csg256")
    n = wl.n
    lab3 = partition(Geometry(n, n, n, wl.angles, n, vial_radius=wl.vial_radius), wl.target, wl.band_width)
    g2 = Geometry(n, n, 1, wl.angles, n, vial_radius=wl.vial_radius)
    tz = np.ascontiguousarray(wl.target[:, :, z:z + 1])
    sep, ops = build_lp(g2, tz, CaseParams(case=1, tol_lo=0.0, tol_hi=10.0, band_width=wl.band_width))
    c2, ops2 = build_lp(g2, tz, CaseParams(case=2, inhibit_ratio=r, band_width=wl.band_width))
    # the slice's rows of the 3-D LP: its gel (same) and the band of the 3-D part
    sep.labels = lab3[:, :, z].ravel().astype(np.uint8)
    c2.labels = lab3[:, :, z].ravel().astype(np.uint8)
    assert c2.f_crit == pytest.approx(r * float(wl.target[wl.target > 0].min()))
    data = pdhg.certificate_data(c2, ops2)
    res, certified = None, False
    for _ in range(8):
        kw = {}
        if res is not None:
            kw = dict(start=(res["y"], res["u"], res["v"]), dual_start=(res["lam_up"], res["lam_lo"]),
                      omega0=res["omega"])
        res = pdhg.solve(sep, ops, kkt_tol=1e-7, max_iter=1024, **kw)
        if pdhg.certificate(c2, ops2, res["lam_up"], res["lam_lo"], *data):
            certified = True
            break
    assert certified
    assert res["obj"] > r
