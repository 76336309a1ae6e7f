"""Host logic of two_stage_solve (Sec. 3.2) with the library calls faked (CPU only):
the stage-2 ratio is u~* (1 + slack), stage 2 starts from the stage-1 point
scaled by 1 / r on the device (sipo_set_primal_from), stage 2 is skipped when
stage 1 is not optimal, and both contexts are released even when stage 2
fails."""
import numpy as np
import pytest

from paper_2604_08997_gb300 import two_stage
from paper_2604_08997_gb300._abi import SIPO_CASE1, SIPO_CASE2, SIPO_F64, SIPO_ITER_LIMIT, SIPO_OPTIMAL


class Fake:
    def __init__(self, u1=0.5, status1=SIPO_OPTIMAL, fail2=False):
        self.u1, self.status1, self.fail2 = u1, status1, fail2
        self.created, self.destroyed, self.started = [], [], []

    def create(self, geometry, f_T, case, tolerances):
        h = len(self.created)
        self.created.append((case, tolerances))
        return h

    def solve(self, ctx, y_out=None):
        case, _ = self.created[ctx]
        if case["kase"] == SIPO_CASE1:
            return {"status": self.status1, "u": self.u1, "pobj": self.u1}
        if self.fail2:
            raise RuntimeError("stage 2 failed")
        return {"status": SIPO_OPTIMAL, "pobj": 1.2}

    def set_primal_from(self, dst, src, scale=1.0, u=-1.0, v=-1.0):
        assert src not in self.destroyed and dst not in self.destroyed
        self.started.append((dst, src, scale))

    def destroy(self, ctx):
        self.destroyed.append(ctx)


def _patch(monkeypatch, f):
    for name, fn in (("sipo_create", f.create), ("sipo_solve", f.solve),
                     ("sipo_set_primal_from", f.set_primal_from), ("sipo_destroy", f.destroy)):
        monkeypatch.setattr(two_stage, name, fn)


GEO = dict(nx=4, ny=4, nz=2, angles=np.zeros(3), n_det=5)


def test_ratio_and_start(monkeypatch):
    fake = Fake()
    _patch(monkeypatch, fake)
    out = two_stage.two_stage_solve(GEO, np.ones((4, 4, 2), np.float32), tol_lo=0.1, tol_hi=0.2,
                                    band_width=3, tolerances=dict(storage=SIPO_F64), slack=0.25)
    r = 0.5 * 1.25
    assert out["ratio"] == r and out["stage2"]["pobj"] == 1.2
    c1, c2 = fake.created[0][0], fake.created[1][0]
    assert c1 == dict(kase=SIPO_CASE1, tol_lo=0.1, tol_hi=0.2, band_width=3)
    assert c2 == dict(kase=SIPO_CASE2, inhibit_ratio=r, band_width=3)
    assert fake.created[1][1] == dict(storage=SIPO_F64)
    assert fake.started == [(1, 0, 1.0 / r)]
    assert sorted(fake.destroyed) == [0, 1]


def test_cold_stage2(monkeypatch):
    fake = Fake()
    _patch(monkeypatch, fake)
    two_stage.two_stage_solve(GEO, np.ones((4, 4, 2), np.float32), warm=False)
    assert fake.started == [] and sorted(fake.destroyed) == [0, 1]


def test_stage2_skipped_unless_stage1_optimal(monkeypatch):
    f = Fake(status1=SIPO_ITER_LIMIT)
    _patch(monkeypatch, f)
    out = two_stage.two_stage_solve(GEO, np.ones((4, 4, 2), np.float32))
    assert out["stage2"] is None and out["ratio"] is None and len(f.created) == 1 and f.destroyed == [0]


def test_contexts_released_when_stage2_fails(monkeypatch):
    f = Fake(fail2=True)
    _patch(monkeypatch, f)
    with pytest.raises(RuntimeError):
        two_stage.two_stage_solve(GEO, np.ones((4, 4, 2), np.float32))
    assert sorted(f.destroyed) == [0, 1]
