"""The C-ABI library loads and exports every symbol include/sipo.h declares (CPU only).

No compute call is made: only argument validation that fails before any
device work.
"""
import ctypes
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_2604_08997_gb300.build import build
    from paper_2604_08997_gb300 import _abi
    build()
    return _abi.load()


def _declared():
    text = open(os.path.join(ROOT, "include", "sipo.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(sipo_[a-z_]+)\s*\(", text)))


def test_header_declares_the_boundary():
    names = _declared()
    for required in ("sipo_create", "sipo_solve", "sipo_project", "sipo_backproject",
                     "sipo_destroy"):
        assert required in names


def test_every_declared_symbol_is_exported(lib):
    from paper_2604_08997_gb300 import _abi
    for name in _declared():
        assert hasattr(lib, name), name
        assert name in _abi.SIGNATURES, f"binding lacks {name}"


def test_invalid_arguments_fail_before_device_work(lib):
    from paper_2604_08997_gb300 import _abi
    ang = np.zeros(4)
    g = _abi.sipo_geometry()
    g.nx, g.ny, g.nz, g.n_angles, g.n_det = 0, 8, 1, 4, 9
    g.angles = ang.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
    cp = _abi.sipo_case_params(0, 1.0, 1.0, 0.05, 0.05, 0.8, 2)
    tl = _abi.sipo_tolerances(1e-4, 100, 64, 0, -1, 0.0)
    tgt = np.ones(64, np.float32)
    out = ctypes.c_void_p()
    rc = lib.sipo_create(ctypes.byref(g), ctypes.c_void_p(tgt.ctypes.data), 0, ctypes.byref(cp),
                         ctypes.byref(tl), None, ctypes.byref(out))
    assert rc == -1
    assert b"positive" in lib.sipo_last_error()
    g.nx = 8
    g.mu = 0.1                                   # attenuation without a vial
    rc = lib.sipo_create(ctypes.byref(g), ctypes.c_void_p(tgt.ctypes.data), 0, ctypes.byref(cp),
                         ctypes.byref(tl), None, ctypes.byref(out))
    assert rc == -1 and b"vial" in lib.sipo_last_error()
    g.mu = 0.0
    cp.kase = 7
    rc = lib.sipo_create(ctypes.byref(g), ctypes.c_void_p(tgt.ctypes.data), 0, ctypes.byref(cp),
                         ctypes.byref(tl), None, ctypes.byref(out))
    assert rc == -1
    # non-finite or out-of-range case parameters
    inf, nan = float("inf"), float("nan")
    for kase, w1, w2, lo, hi, r in ((0, inf, 1.0, 0.05, 0.05, 0.8), (0, 1.0, nan, 0.05, 0.05, 0.8),
                                    (1, 1.0, 1.0, 0.05, inf, 0.8), (1, 1.0, 1.0, 1.0, 0.05, 0.8),
                                    (2, 1.0, 1.0, 0.05, 0.05, inf), (2, 1.0, 1.0, 0.05, 0.05, 0.0)):
        bad = _abi.sipo_case_params(kase, w1, w2, lo, hi, r, 2)
        rc = lib.sipo_create(ctypes.byref(g), ctypes.c_void_p(tgt.ctypes.data), 0, ctypes.byref(bad),
                             ctypes.byref(tl), None, ctypes.byref(out))
        assert rc == -1, (kase, w1, w2, lo, hi, r)
    # the problem-size limit (2^34 voxels) is checked before any allocation
    g.nx, g.ny, g.nz = 1 << 12, 1 << 12, 1 << 11
    rc = lib.sipo_create(ctypes.byref(g), ctypes.c_void_p(tgt.ctypes.data), 0, ctypes.byref(cp),
                         ctypes.byref(tl), None, ctypes.byref(out))
    assert rc == -1 and b"too large" in lib.sipo_last_error()
    assert lib.sipo_destroy(None) == 0
    assert lib.sipo_phase_count() >= 3
    assert lib.sipo_phase_name(0) == b"scalar_step"


def test_new_entries_validate_before_device_work(lib):
    """Bounded creation, the response map and metrics, the state import /
    export and the primal start refuse bad arguments before any CUDA call."""
    from paper_2604_08997_gb300 import _abi
    ang = np.zeros(4)
    g = _abi.sipo_geometry()
    g.nx, g.ny, g.nz, g.n_angles, g.n_det = 8, 8, 1, 4, 9
    g.angles = ang.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
    tl = _abi.sipo_tolerances(1e-4, 100, 64, 0, -1, 0.0)
    tgt = np.ones(64, np.float32)
    p = ctypes.c_void_p(tgt.ctypes.data)
    out = ctypes.c_void_p()
    cp2 = _abi.sipo_case_params(2, 1.0, 1.0, 0.05, 0.05, 0.8, 2)
    rc = lib.sipo_create_bounded(ctypes.byref(g), p, p, p, 0, ctypes.byref(cp2), ctypes.byref(tl), None,
                                 ctypes.byref(out))
    assert rc == -1 and b"Case-1" in lib.sipo_last_error()
    cp1 = _abi.sipo_case_params(1, 1.0, 1.0, 0.05, 0.05, 0.8, 2)
    rc = lib.sipo_create_bounded(ctypes.byref(g), p, None, p, 0, ctypes.byref(cp1), ctypes.byref(tl), None,
                                 ctypes.byref(out))
    assert rc == -1 and b"null" in lib.sipo_last_error()
    for bad in ((0.0, 0.0, 8.0, 0.7, 0.5), (0.0, 1.0, -1.0, 0.7, 0.5), (0.0, 1.0, 8.0, 0.0, 0.5),
                (float("nan"), 1.0, 8.0, 0.7, 0.5)):
        r = _abi.sipo_response(*bad)
        rc = lib.sipo_response_map(ctypes.byref(r), p, p, 64, 1.0, 1, None)
        assert rc == -1 and b"response model" in lib.sipo_last_error()
        res = _abi.sipo_response_result()
        rc = lib.sipo_response_metrics(None, ctypes.byref(r), p, 0, 0.0, ctypes.byref(res))
        assert rc == -1
    good = _abi.sipo_response(0.0, 1.0, 8.0, 0.7, 0.5)
    assert lib.sipo_response_map(ctypes.byref(good), p, p, 0, 1.0, 1, None) == 0     # empty: no work
    rc = lib.sipo_response_map(ctypes.byref(good), p, p, 64, float("inf"), 1, None)
    assert rc == -1 and b"scale" in lib.sipo_last_error()
    rc = lib.sipo_response_map(ctypes.byref(good), None, p, 64, 1.0, 1, None)
    assert rc == -1 and b"null" in lib.sipo_last_error()
    sc = (ctypes.c_double * 4)()
    assert lib.sipo_get_state(None, None, None, None, 0, sc) == -1
    assert lib.sipo_set_state(None, p, p, p, 0, sc) == -1
    assert lib.sipo_set_primal(None, p, 0, -1.0, -1.0) == -1
    assert b"null" in lib.sipo_last_error()
    assert lib.sipo_set_primal_from(None, None, 1.0, -1.0, -1.0) == -1
    assert b"null" in lib.sipo_last_error()
    fake = ctypes.c_void_p(1)
    assert lib.sipo_set_primal_from(fake, fake, 1.0, -1.0, -1.0) == -1
    assert b"same context" in lib.sipo_last_error()
    # probe and race: null, repeated contexts and a non-positive probe period
    # are refused on the pointers alone
    res, res2 = _abi.sipo_result(), _abi.sipo_result()
    cert, sl = ctypes.c_int(0), ctypes.c_int(0)
    a, b, c = ctypes.c_void_p(1), ctypes.c_void_p(2), ctypes.c_void_p(3)
    refs = (ctypes.byref(res), ctypes.byref(cert), ctypes.byref(sl))
    assert lib.sipo_solve_probe(None, b, 128, *refs) == -1 and b"null" in lib.sipo_last_error()
    assert lib.sipo_solve_probe(a, a, 128, *refs) == -1 and b"same" in lib.sipo_last_error()
    assert lib.sipo_solve_probe(a, b, 0, *refs) == -1 and b"probe_every" in lib.sipo_last_error()
    rrefs = (ctypes.byref(res), ctypes.byref(res2), ctypes.byref(cert), ctypes.byref(sl))
    assert lib.sipo_solve_race(a, b, None, 128, *rrefs) == -1 and b"null" in lib.sipo_last_error()
    assert lib.sipo_solve_race(a, b, c, 128, ctypes.byref(res), None, ctypes.byref(cert),
                               ctypes.byref(sl)) == -1
    for x, y, z in ((a, a, c), (a, b, a), (a, b, b)):
        assert lib.sipo_solve_race(x, y, z, 128, *rrefs) == -1 and b"distinct" in lib.sipo_last_error()
    assert lib.sipo_solve_race(a, b, c, 0, *rrefs) == -1 and b"probe_every" in lib.sipo_last_error()
    n_out = ctypes.c_uint(7)
    for budget, threads, outp in ((0, 32, ctypes.byref(n_out)), (1000, 0, ctypes.byref(n_out)),
                                  (1000, 1025, ctypes.byref(n_out)), (1000, 32, None)):
        assert lib.sipo_wait_selftest(budget, 0, threads, outp) == -1
        assert b"wait self-test" in lib.sipo_last_error()


def test_noalloc_wrapper_refuses_mismatched_buffers():
    """The scratch-free metrics wrapper checks dtypes, sizes and locations on the
    host; each mismatch raises before the library is loaded or called."""
    torch = pytest.importorskip("torch")
    from paper_2604_08997_gb300 import _abi
    d = torch.zeros(8)
    lab = torch.zeros(8, dtype=torch.uint8)
    f = torch.ones(8)
    cases = [
        (d, lab.to(torch.int32), f, "labels must be uint8"),
        (d, lab, f.double(), "f_T must be float32"),
        (d, lab[:7], f, "labels has 7 elements"),
        (d, lab, f[:6], "f_T has 6 elements"),
        (d, lab, f, "must be device tensors"),
    ]
    for dose, labels, ft, msg in cases:
        with pytest.raises(ValueError, match=msg):
            _abi.sipo_dose_metrics_noalloc(dose, labels, ft, 1.0, 1.0)
