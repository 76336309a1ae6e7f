"""Case 2 with its feasibility settled first (Secs. 2.7.1-2.7.2, infeasibility as
a diagnostic).

Case 2 at an inhibition ratio r asks for band dose d <= 1 while every gel
voxel gets d >= f_T / (r min f_T) (Eqs. 40-45).  Whether such a dose exists
is itself an LP, the separation LP: minimise the band maximum u~ subject to
f_T / min f_T <= d on gel.  Case 2 at r is feasible exactly when its optimum
u~* is at most r.  The separation LP is Case 1 of the same part (Eqs. 32-37)
with tol_lo = 0 and a loose upper tolerance (gel dose up to (1 + tol_hi)
times its target, tol_hi = 10 by default, far above any optimal spread), so
it is always feasible and bounded and the PDHG converges on it where the
Case-2 iterates of an infeasible ratio only drift.

The workflow solves it while testing, every `probe_every` iterations, its
current dual point as a Farkas ray of Case 2 at r (sipo_solve_probe runs the
library's bound-based test, slice by slice where the PSF allows).  A ray is a
certificate by itself, whatever the accuracy of the iterate that gave it, so
the first one that passes ends the workflow with PRIMAL_INFEASIBLE.  Passing
duals can come and go between restarts (on the blurred 256^3 part one passes
at iteration 1280 and none at 2048 or 3072), so the probes are frequent: every
128 iterations by default, each about one projection.  If the
separation LP ends instead with u~ <= r, its primal point over r satisfies
every Case-2 row (up to its primal residual) and starts the Case-2 solve
(sipo_set_primal_from), as the two-stage design of Sec. 3.2 does with a
Case-1 point; otherwise Case 2 runs from zero.  Host orchestration only: every step runs in libsipo.
"""
from __future__ import annotations

from ._abi import (SIPO_CASE1, SIPO_CASE2, SIPO_OPTIMAL, SIPO_PRIMAL_INFEASIBLE, sipo_create, sipo_destroy,
                   sipo_set_primal_from, sipo_solve, sipo_solve_probe)


def case2_with_separation(geometry: dict, f_T, ratio: float, band_width: int = 10,
                          tolerances: dict | None = None, separation_tolerances: dict | None = None,
                          probe_every: int = 128, tol_hi: float = 10.0) -> dict:
    """Case 2 at inhibition ratio `ratio`, preceded by the separation LP.

    Returns {"separation": result of the separation LP, "ratio_bound": its
    u~ (the best band-to-gel ratio found), "certified": bool, "cert_slice":
    int, "case2": result of the Case-2 solve or None, "status": the Case-2
    status (SIPO_PRIMAL_INFEASIBLE when certified)}.  `separation_tolerances`
    defaults to `tolerances`.
    """
    tol = dict(tolerances or {})
    tol_sep = dict(separation_tolerances if separation_tolerances is not None else tol)
    sep = sipo_create(geometry, f_T, dict(kase=SIPO_CASE1, tol_lo=0.0, tol_hi=tol_hi, band_width=band_width),
                      tol_sep)
    ctx2 = None
    try:
        ctx2 = sipo_create(geometry, f_T, dict(kase=SIPO_CASE2, inhibit_ratio=ratio, band_width=band_width), tol)
        rs, cert, sl = sipo_solve_probe(sep, ctx2, probe_every)
        out = {"separation": rs, "ratio_bound": rs["pobj"], "certified": cert, "cert_slice": sl,
               "case2": None, "status": None}
        if cert:
            out["status"] = SIPO_PRIMAL_INFEASIBLE
            return out
        if rs["pobj"] <= ratio:
            # band d <= u~ <= r and gel d >= f_T / min f_T: over r, a Case-2
            # point (up to the separation's primal residual if it stopped early)
            sipo_set_primal_from(ctx2, sep, 1.0 / ratio)
        r2 = sipo_solve(ctx2)
        out.update(case2=r2, status=r2["status"])
        return out
    finally:
        sipo_destroy(sep)
        if ctx2 is not None:
            sipo_destroy(ctx2)
