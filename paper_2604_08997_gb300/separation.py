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
current dual point as a Farkas ray of Case 2 at r (the library's bound-based
test, slice by slice where the PSF allows).  A ray is a
certificate by itself, whatever the accuracy of the iterate that gave it, so
the first one that passes ends the workflow with PRIMAL_INFEASIBLE.  Passing
duals can come and go between restarts (on the blurred 256^3 part one passes
at iteration 1280 and none at 2048 or 3072), so the probes are frequent: every
128 iterations by default, each about one projection.  In the sequential
form, if the separation LP ends instead with u~ <= r, its primal point over r satisfies
every Case-2 row (up to its primal residual) and starts the Case-2 solve
(sipo_set_primal_from), as the two-stage design of Sec. 3.2 does with a
Case-1 point; otherwise Case 2 runs from zero.

That sequence (race=False) is slow where r is feasible: on the 256^3 part at
r = 0.85 the separation LP had not reached KKT 1e-4 after 16384 iterations,
and Case 2 started from its scaled point had not after 2048, where from zero
it does in 1344 (26 s in all, against 1.9 s for Case 2 alone).  So by
default (race=True) Case 2 itself is solved at the same time as the
separation LP, on a stream of its own (sipo_solve_race): a feasible r ends
with the Case-2 optimum, an infeasible one with the first certificate of the
probes, whichever comes first.  Host orchestration only: every step runs in
libsipo.
"""
from __future__ import annotations

from ._abi import (SIPO_CASE1, SIPO_CASE2, SIPO_PRIMAL_INFEASIBLE, sipo_create, sipo_destroy,
                   sipo_set_primal_from, sipo_solve, sipo_solve_probe, sipo_solve_race)


def case2_with_separation(geometry: dict, f_T, ratio: float, band_width: int = 10,
                          tolerances: dict | None = None, separation_tolerances: dict | None = None,
                          probe_every: int = 128, tol_hi: float = 10.0, race: bool = True) -> dict:
    """Case 2 at inhibition ratio `ratio`, preceded by the separation LP.

    Returns {"separation": result of the separation LP, "ratio_bound": its
    u~ (the best band-to-gel ratio found), "certified": bool, "cert_slice":
    int, "case2": result of the Case-2 solve (None when the sequential
    form certified first), "status": the Case-2 status (SIPO_PRIMAL_INFEASIBLE
    when certified)}.  `separation_tolerances` defaults to `tolerances`;
    `race` picks the concurrent form (True) or the sequential one.
    """
    tol = dict(tolerances or {})
    tol_sep = dict(separation_tolerances if separation_tolerances is not None else tol)
    sep = sipo_create(geometry, f_T, dict(kase=SIPO_CASE1, tol_lo=0.0, tol_hi=tol_hi, band_width=band_width),
                      tol_sep)
    ctx2 = rival = None
    case2 = dict(kase=SIPO_CASE2, inhibit_ratio=ratio, band_width=band_width)
    try:
        ctx2 = sipo_create(geometry, f_T, case2, tol)
        if race:
            # a probe resets its target's solver state: the solved Case 2 is a
            # context of its own
            rival = sipo_create(geometry, f_T, case2, tol)
            rs, r2, cert, sl = sipo_solve_race(sep, ctx2, rival, probe_every)
            return {"separation": rs, "ratio_bound": rs["pobj"], "certified": cert, "cert_slice": sl,
                    "case2": r2, "status": SIPO_PRIMAL_INFEASIBLE if cert else r2["status"]}
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
        for c in (ctx2, rival):
            if c is not None:
                sipo_destroy(c)
