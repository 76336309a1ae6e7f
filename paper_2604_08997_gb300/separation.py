"""Case 2 with its feasibility settled first (Secs. 2.6-2.7.2, infeasibility as
a diagnostic).

Case 2 at an inhibition ratio r asks for band dose d <= 1 while every gel
voxel gets d >= f_T / (r min f_T) (Eqs. 40-45).  Whether such a dose exists
is itself an LP: the general form of Eqs. 19-24 with weights w1 = 1, w2 = 0
on the same part minimises u~ subject to band d <= u~ and gel d >= f_T /
min f_T, so its optimum u~* is the smallest band-to-gel dose ratio any
projection reaches, and Case 2 at r is feasible exactly when u~* <= r.  That
LP is always feasible and bounded, so the PDHG converges on it where the
Case-2 iterates of an infeasible ratio only drift.

The workflow solves it first.  If u~* > r, its optimal dual point is a Farkas
ray of Case 2 at r (sipo_farkas_from runs the library's bound-based test on
it, slice by slice), which certifies PRIMAL_INFEASIBLE.  Otherwise its primal
point, scaled by 1 / r, satisfies every Case-2 row and starts the Case-2 solve
(sipo_set_primal_from), as the two-stage design of Sec. 3.2 does with a
Case-1 point.  Host orchestration only: every step runs in libsipo.
"""
from __future__ import annotations

from ._abi import (SIPO_CASE2, SIPO_GENERAL, SIPO_OPTIMAL, SIPO_PRIMAL_INFEASIBLE, sipo_create,
                   sipo_destroy, sipo_farkas_from, sipo_set_primal_from, sipo_solve)


def case2_with_separation(geometry: dict, f_T, ratio: float, band_width: int = 10,
                          tolerances: dict | None = None, separation_tolerances: dict | None = None) -> dict:
    """Case 2 at inhibition ratio `ratio`, preceded by the separation LP.

    Returns {"separation": result of the general form (w1 = 1, w2 = 0),
    "ratio_bound": its optimum u~*, "certified": bool, "cert_slice": int,
    "case2": result of the Case-2 solve or None, "status": the Case-2 status
    (SIPO_PRIMAL_INFEASIBLE when certified)}.  `separation_tolerances`
    defaults to `tolerances`.
    """
    tol = dict(tolerances or {})
    tol_sep = dict(separation_tolerances if separation_tolerances is not None else tol)
    sep = sipo_create(geometry, f_T, dict(kase=SIPO_GENERAL, w1=1.0, w2=0.0, band_width=band_width), tol_sep)
    ctx2 = None
    try:
        rs = sipo_solve(sep)
        out = {"separation": rs, "ratio_bound": rs["pobj"], "certified": False, "cert_slice": -1,
               "case2": None, "status": None}
        ctx2 = sipo_create(geometry, f_T, dict(kase=SIPO_CASE2, inhibit_ratio=ratio, band_width=band_width), tol)
        if rs["pobj"] > ratio:
            cert, sl = sipo_farkas_from(ctx2, sep)
            if cert:
                out.update(certified=True, cert_slice=sl, status=SIPO_PRIMAL_INFEASIBLE)
                return out
        elif rs["status"] == SIPO_OPTIMAL:
            # band d <= u~* <= r and gel d >= f_T / min f_T: over r, a Case-2 point
            sipo_set_primal_from(ctx2, sep, 1.0 / ratio)
        r2 = sipo_solve(ctx2)
        out.update(case2=r2, status=r2["status"])
        return out
    finally:
        sipo_destroy(sep)
        if ctx2 is not None:
            sipo_destroy(ctx2)
