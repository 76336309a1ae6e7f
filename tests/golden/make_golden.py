"""Writes the stored expected values under tests/golden/ (calls only oracle/).

disc64_case1.json: optimum of the Case-1 LP (Eqs. 32-37, delta = 0.05) on the
64x64 / 96-angle / 91-bin three-disc slice, from the oracle's restarted PDHG
run to a relative KKT error of 1e-7 (objective accurate to ~1e-7 relative).
"""
import json
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

from oracle import pdhg  # noqa: E402
from oracle.lp import CaseParams, build_lp  # noqa: E402
from oracle.operators import Geometry  # noqa: E402
from synthetic.targets import workload  # noqa: E402


def main():
    wl = workload("disc64")
    lp, ops = build_lp(Geometry(64, 64, 1, wl.angles, 91), wl.target,
                       CaseParams(case=1, tol_lo=0.05, tol_hi=0.05, band_width=10))
    res = pdhg.solve(lp, ops, kkt_tol=1e-7, max_iter=400000)
    out = dict(workload="disc64 (64x64, 96 angles over [0, pi), 91 bins, 3 discs, seed 1)",
               case="Case 1, tol_lo = tol_hi = 0.05, band width 10",
               source="oracle.pdhg.solve, kkt_tol 1e-7",
               status=int(res["status"]), iterations=int(res["iters"]),
               objective=res["obj"], kkt=res["info"]["kkt"],
               metrics={k: float(v) for k, v in res["metrics"].items()})
    with open(os.path.join(HERE, "disc64_case1.json"), "w") as f:
        json.dump(out, f, indent=1)
    print(out)


if __name__ == "__main__":
    main()
