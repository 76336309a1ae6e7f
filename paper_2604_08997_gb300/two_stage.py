"""Two-stage design (Sec. 3.2): Case 1 fixes the process bound, Case 2 then
recovers target conformity at that bound.

Stage 1 solves the target-bounded LP (Case 1): gel dose within
[(1 - d_lo) f_T, (1 + d_hi) f_T] up to scale, minimum band dose ratio u~*
relative to f_crit = (1 - d_lo) min f_T.  Its solution separates gel from
band by min-gel / max-band >= 1 / u~*.

Stage 2 solves the dose-shaping LP (Case 2) with the inhibition ratio
r = u~* (1 + slack), i.e. band dose <= r min f_T while gel dose >= f_T: the
same separation, now with the gel spread v~ (DTVR) minimised.  The stage-1
dose scaled by 1 / (1 - d_lo) satisfies every stage-2 row for any r >= u~*:
in normalised units (dose / f_crit of each stage) that point is y2 = y1 / r,
so stage 2 is feasible by construction, its optimum v~* is at most that
point's spread (<= (1 + d_hi) / (1 - d_lo)), and stage 2 may start from it
instead of from zero.

Host orchestration only: both solves run in libsipo, and the stage-1 point
goes to stage 2 on the device (`sipo_set_primal_from` with scale 1 / r).
"""
from __future__ import annotations

from ._abi import (SIPO_CASE1, SIPO_CASE2, SIPO_OPTIMAL, sipo_create, sipo_destroy, sipo_set_primal_from,
                   sipo_solve)


def two_stage_solve(geometry: dict, f_T, tol_lo: float = 0.05, tol_hi: float = 0.05,
                    band_width: int = 10, tolerances: dict | None = None,
                    tolerances2: dict | None = None, slack: float = 0.0,
                    warm: bool = True) -> dict:
    """Stage 1 (Case 1 at tolerance tol_lo / tol_hi), then stage 2 (Case 2 at
    r = u~*(1 + slack)), started from the rescaled stage-1 point when `warm`.

    Returns {"stage1": result, "stage2": result or None, "ratio": r or None}.
    Stage 2 runs only when stage 1 is optimal.  `tolerances2` defaults to
    `tolerances`.
    """
    tol1 = dict(tolerances or {})
    tol2 = dict(tolerances2 if tolerances2 is not None else tol1)
    c1 = dict(kase=SIPO_CASE1, tol_lo=tol_lo, tol_hi=tol_hi, band_width=band_width)
    ctx1 = sipo_create(geometry, f_T, c1, tol1)
    ctx2 = None
    try:
        res1 = sipo_solve(ctx1)
        out = {"stage1": res1, "stage2": None, "ratio": None}
        if res1["status"] != SIPO_OPTIMAL or not res1["u"] > 0:
            return out
        r = float(res1["u"]) * (1.0 + slack)
        out["ratio"] = r
        c2 = dict(kase=SIPO_CASE2, inhibit_ratio=r, band_width=band_width)
        ctx2 = sipo_create(geometry, f_T, c2, tol2)
        if warm:
            # the stage-1 dose over (1 - d_lo), in stage-2 normalised units
            sipo_set_primal_from(ctx2, ctx1, 1.0 / r)
        out["stage2"] = sipo_solve(ctx2)
        return out
    finally:
        sipo_destroy(ctx1)
        if ctx2 is not None:
            sipo_destroy(ctx2)
