"""Host logic of case2_with_separation with the library calls faked (CPU only):
the separation LP is Case 1 of the same part with tol_lo = 0 and a loose
upper tolerance, solved with Farkas probes of the Case-2 context; a
certificate ends the workflow as PRIMAL_INFEASIBLE; a separation value at or
below the ratio starts Case 2 from the separation point scaled by 1 / r;
otherwise Case 2 runs from zero; contexts are always released."""
from paper_2604_08997_gb300 import separation
from paper_2604_08997_gb300._abi import (SIPO_CASE1, SIPO_CASE2, SIPO_ITER_LIMIT, SIPO_OPTIMAL,
                                         SIPO_PRIMAL_INFEASIBLE)


class Fake:
    def __init__(self, bound, certified=False, sep_status=SIPO_OPTIMAL):
        self.bound, self.certified, self.sep_status = bound, certified, sep_status
        self.created, self.destroyed, self.calls = [], [], []

    def create(self, geometry, f_T, case, tolerances):
        self.created.append(case)
        return len(self.created) - 1

    def probe(self, ctx, target, probe_every=1024):
        self.calls.append(("probe", ctx, target, probe_every))
        return {"status": self.sep_status, "pobj": self.bound}, self.certified, 7 if self.certified else -1

    def solve(self, ctx):
        self.calls.append(("solve", ctx))
        return {"status": SIPO_OPTIMAL, "pobj": 1.1}

    def primal_from(self, dst, src, scale=1.0, u=-1.0, v=-1.0):
        self.calls.append(("start", dst, src, scale))

    def destroy(self, ctx):
        self.destroyed.append(ctx)


def _run(monkeypatch, fake, ratio=0.8):
    for name, fn in (("sipo_create", fake.create), ("sipo_solve", fake.solve), ("sipo_solve_probe", fake.probe),
                     ("sipo_set_primal_from", fake.primal_from), ("sipo_destroy", fake.destroy)):
        monkeypatch.setattr(separation, name, fn)
    return separation.case2_with_separation({}, None, ratio, band_width=3, tolerances={"kkt_tol": 1e-4},
                                            probe_every=512)


def test_certified_infeasible(monkeypatch):
    f = Fake(bound=0.83, certified=True, sep_status=SIPO_ITER_LIMIT)
    out = _run(monkeypatch, f)
    assert f.created[0] == dict(kase=SIPO_CASE1, tol_lo=0.0, tol_hi=10.0, band_width=3)
    assert f.created[1] == dict(kase=SIPO_CASE2, inhibit_ratio=0.8, band_width=3)
    assert ("probe", 0, 1, 512) in f.calls
    assert out["status"] == SIPO_PRIMAL_INFEASIBLE and out["certified"] and out["cert_slice"] == 7
    assert out["ratio_bound"] == 0.83 and out["case2"] is None and ("solve", 1) not in f.calls
    assert sorted(f.destroyed) == [0, 1]


def test_uncertified_bound_solves_case2_from_zero(monkeypatch):
    f = Fake(bound=0.83)
    out = _run(monkeypatch, f)
    assert not out["certified"] and out["status"] == SIPO_OPTIMAL
    assert not any(c[0] == "start" for c in f.calls) and ("solve", 1) in f.calls


def test_feasible_ratio_starts_from_the_scaled_point(monkeypatch):
    f = Fake(bound=0.7)
    out = _run(monkeypatch, f)
    assert ("start", 1, 0, 1.0 / 0.8) in f.calls
    assert out["status"] == SIPO_OPTIMAL and out["case2"]["pobj"] == 1.1


def test_unconverged_separation_below_the_ratio_still_starts_case2(monkeypatch):
    f = Fake(bound=0.7, sep_status=SIPO_ITER_LIMIT)
    out = _run(monkeypatch, f)
    assert ("start", 1, 0, 1.0 / 0.8) in f.calls and out["status"] == SIPO_OPTIMAL
