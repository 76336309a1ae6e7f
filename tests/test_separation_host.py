"""Host logic of case2_with_separation with the library calls faked (CPU only):
the separation LP is Case 1 of the same part with tol_lo = 0 and a loose
upper tolerance, solved with Farkas probes of a Case-2 context.  Sequential
form: a certificate ends the workflow as PRIMAL_INFEASIBLE; a separation
value at or below the ratio starts Case 2 from the separation point scaled by
1 / r; otherwise Case 2 runs from zero.  Concurrent form: a second Case-2
context is solved beside the separation LP and its status is the workflow's
unless a probe certified.  Contexts are always released."""
from paper_2604_08997_gb300 import separation
from paper_2604_08997_gb300._abi import (SIPO_CASE1, SIPO_CASE2, SIPO_ITER_LIMIT, SIPO_OPTIMAL,
                                         SIPO_PRIMAL_INFEASIBLE)


class Fake:
    def __init__(self, bound, certified=False, sep_status=SIPO_OPTIMAL, rival_status=SIPO_OPTIMAL):
        self.bound, self.certified, self.sep_status = bound, certified, sep_status
        self.rival_status = rival_status
        self.created, self.destroyed, self.calls = [], [], []

    def create(self, geometry, f_T, case, tolerances):
        self.created.append(case)
        return len(self.created) - 1

    def probe(self, ctx, target, probe_every=1024):
        self.calls.append(("probe", ctx, target, probe_every))
        return {"status": self.sep_status, "pobj": self.bound}, self.certified, 7 if self.certified else -1

    def race(self, ctx, target, rival, probe_every=1024):
        self.calls.append(("race", ctx, target, rival, probe_every))
        status = SIPO_ITER_LIMIT if self.certified else self.rival_status
        return ({"status": self.sep_status, "pobj": self.bound}, {"status": status, "pobj": 1.2},
                self.certified, 7 if self.certified else -1)

    def solve(self, ctx):
        self.calls.append(("solve", ctx))
        return {"status": SIPO_OPTIMAL, "pobj": 1.1}

    def primal_from(self, dst, src, scale=1.0, u=-1.0, v=-1.0):
        self.calls.append(("start", dst, src, scale))

    def destroy(self, ctx):
        self.destroyed.append(ctx)


def _run(monkeypatch, fake, ratio=0.8, race=False):
    for name, fn in (("sipo_create", fake.create), ("sipo_solve", fake.solve), ("sipo_solve_probe", fake.probe),
                     ("sipo_solve_race", fake.race), ("sipo_set_primal_from", fake.primal_from),
                     ("sipo_destroy", fake.destroy)):
        monkeypatch.setattr(separation, name, fn)
    return separation.case2_with_separation({}, None, ratio, band_width=3, tolerances={"kkt_tol": 1e-4},
                                            probe_every=512, race=race)


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


def test_race_certified(monkeypatch):
    f = Fake(bound=0.83, certified=True, sep_status=SIPO_ITER_LIMIT)
    out = _run(monkeypatch, f, race=True)
    case2 = dict(kase=SIPO_CASE2, inhibit_ratio=0.8, band_width=3)
    assert f.created == [dict(kase=SIPO_CASE1, tol_lo=0.0, tol_hi=10.0, band_width=3), case2, case2]
    assert ("race", 0, 1, 2, 512) in f.calls
    assert not any(c[0] in ("solve", "start", "probe") for c in f.calls)
    assert out["status"] == SIPO_PRIMAL_INFEASIBLE and out["certified"] and out["cert_slice"] == 7
    assert out["case2"]["status"] == SIPO_ITER_LIMIT and out["ratio_bound"] == 0.83
    assert sorted(f.destroyed) == [0, 1, 2]


def test_race_takes_the_rival_status(monkeypatch):
    for st in (SIPO_OPTIMAL, SIPO_PRIMAL_INFEASIBLE, SIPO_ITER_LIMIT):
        f = Fake(bound=0.7, sep_status=SIPO_ITER_LIMIT, rival_status=st)
        out = _run(monkeypatch, f, race=True)
        assert not out["certified"] and out["status"] == st and out["case2"]["pobj"] == 1.2
        assert sorted(f.destroyed) == [0, 1, 2]


def test_race_is_the_default(monkeypatch):
    f = Fake(bound=0.7)
    for name, fn in (("sipo_create", f.create), ("sipo_solve_race", f.race), ("sipo_destroy", f.destroy)):
        monkeypatch.setattr(separation, name, fn)
    separation.case2_with_separation({}, None, 0.8)
    assert f.calls and f.calls[0][0] == "race"


def test_contexts_released_when_creation_fails(monkeypatch):
    f = Fake(bound=0.7)
    made = []

    def create(geometry, f_T, case, tolerances):
        if len(made) == 2:
            raise RuntimeError("out of device memory")
        made.append(case)
        return len(made) - 1

    for name, fn in (("sipo_create", create), ("sipo_solve_race", f.race), ("sipo_destroy", f.destroy)):
        monkeypatch.setattr(separation, name, fn)
    try:
        separation.case2_with_separation({}, None, 0.8)
    except RuntimeError:
        pass
    else:
        raise AssertionError("creation failure not raised")
    assert sorted(f.destroyed) == [0, 1]


def test_contexts_released_when_the_race_fails(monkeypatch):
    f = Fake(bound=0.7)

    def race(ctx, target, rival, probe_every=1024):
        raise RuntimeError("sipo error -5: non-finite iterates")

    for name, fn in (("sipo_create", f.create), ("sipo_solve_race", race), ("sipo_destroy", f.destroy)):
        monkeypatch.setattr(separation, name, fn)
    try:
        separation.case2_with_separation({}, None, 0.8)
    except RuntimeError:
        pass
    else:
        raise AssertionError("race failure not raised")
    assert sorted(f.destroyed) == [0, 1, 2]
