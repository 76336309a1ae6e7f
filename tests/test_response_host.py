"""Host logic of the response-domain front end (Sec. 2.1, Eq. 5; Sec. 2.7.1) with
the device calls faked by the oracle's FP64 map on CPU tensors (CPU only):
Case 1 passes M^-1 of m_T, (1 - eps_lo) m_T and (1 + eps_hi) m_T as target and
bounds; Case 2 passes the ratio M^-1(m_crit) / M^-1(min_gel m_T) that the
library computes on the device (faked here by the oracle's map)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle.response import Richards as ORichards
from oracle.response import response_inverse
from paper_2604_08997_gb300 import response as R

MP = (0.0, 1.0, 8.0, 0.7, 0.5)


@pytest.fixture
def fake(monkeypatch):
    calls = {}

    def device(a):
        if isinstance(a, np.ndarray):
            a = torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32))
        return a.to(dtype=torch.float32).contiguous()

    def rmap(M, src, dst, inverse, scale=1.0, stream=None):
        assert inverse
        v = scale * src.double().numpy()
        dst.copy_(torch.from_numpy(response_inverse(ORichards(*M), v)).float())
        return dst

    def create(geometry, f_T, case, tolerances):
        calls["create"] = (f_T.clone(), case)
        return "ctx"

    def create_bounded(geometry, f_T, f_L, f_U, case, tolerances):
        calls["bounded"] = (f_T.clone(), f_L.clone(), f_U.clone(), case)
        return "ctx"

    def ratio(M, m, m_crit, stream=None):
        om = ORichards(*M)
        v = m.double().numpy()
        gmin = float(v[v > M[0]].min())
        return float(response_inverse(om, np.array([m_crit]))[0] / response_inverse(om, np.array([gmin]))[0]), gmin

    monkeypatch.setattr(R, "_device", device)
    monkeypatch.setattr(R, "sipo_response_inhibit_ratio", ratio)
    monkeypatch.setattr(R, "sipo_response_map", rmap)
    monkeypatch.setattr(R, "sipo_create", create)
    monkeypatch.setattr(R, "sipo_create_bounded", create_bounded)
    return calls


def _m():
    m = np.zeros((6, 6, 1), np.float32)
    m[1:3, 1:3] = 0.7
    m[3:5, 3:5] = 0.5
    return m


def test_case1_bounds(fake):
    M = R.Richards(*MP)
    R.response_case1(dict(), _m(), M, eps_lo=0.05, eps_hi=0.1, band_width=3)
    fT, fL, fU, case = fake["bounded"]
    m = _m().astype(np.float64)
    om = ORichards(*MP)
    np.testing.assert_allclose(fT.numpy(), response_inverse(om, m), rtol=1e-6)
    np.testing.assert_allclose(fL.numpy(), response_inverse(om, 0.95 * m), rtol=1e-6)
    np.testing.assert_allclose(fU.numpy(), response_inverse(om, 1.1 * m), rtol=1e-6)
    assert case == dict(band_width=3)
    gel = m > 0
    assert np.all(fL.numpy()[gel] < fT.numpy()[gel]) and np.all(fT.numpy()[gel] < fU.numpy()[gel])


def test_case2_ratio(fake):
    M = R.Richards(*MP)
    R.response_case2(dict(), _m(), M, m_crit=0.33, band_width=2)
    fT, case = fake["create"]
    om = ORichards(*MP)
    want = response_inverse(om, np.array([0.33]))[0] / response_inverse(om, np.array([0.5]))[0]
    assert case["kase"] == 2 and case["band_width"] == 2
    assert abs(case["inhibit_ratio"] - want) <= 1e-6 * want


def test_general(fake):
    R.response_general(dict(), _m(), R.Richards(*MP), w1=2.0, w2=0.5, band_width=4)
    fT, case = fake["create"]
    assert case == dict(kase=0, w1=2.0, w2=0.5, band_width=4)
    assert float(fT.max()) == pytest.approx(float(response_inverse(ORichards(*MP), np.array([0.7]))[0]),
                                            rel=1e-6)
