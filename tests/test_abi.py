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
    assert lib.sipo_destroy(None) == 0
    assert lib.sipo_phase_count() >= 3
    assert lib.sipo_phase_name(0) == b"scalar_step"
