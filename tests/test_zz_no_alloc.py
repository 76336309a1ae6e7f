"""Dose metrics without device allocation (GPU; collected last on purpose).

Some callers of this library may not allocate device memory at all: a print
controller that must not allocate once its real-time loop runs, or code inside
a framework whose caching allocator owns the device-memory budget.
sipo_dose_metrics_noalloc serves them: it repeats the metrics pass that ends
sipo_solve with its partial sums in a static device array of the library.
This file calls it through the C ABI twice in a row and compares both results
with the metrics sipo_solve reported for the same dose field, checks that the
second call leaves the device's free memory unchanged, and that requests above
the array's limit are refused.
"""
import ctypes

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from synthetic.targets import csg_3d, uniform_angles

FP32_TOL = 1e-5
FP64_TOL = 1e-12


@pytest.fixture(scope="module")
def sipo():
    import paper_2604_08997_gb300 as s
    s.build()
    return s


@pytest.mark.parametrize("storage", ["f32", "f64"])
@pytest.mark.parametrize("kase", [1, 2])
def test_noalloc_metrics_match_the_solver(sipo, storage, kase):
    from paper_2604_08997_gb300 import _abi
    n = 32
    tgt = csg_3d(n, vial_radius=15.0, band_width=2, seed=2, feature=(3.0, 10.0))
    ang = uniform_angles(45)
    st, dt, tol = ((sipo.SIPO_F32, torch.float32, FP32_TOL) if storage == "f32"
                   else (sipo.SIPO_F64, torch.float64, FP64_TOL))
    cp = dict(kase=kase, band_width=2, inhibit_ratio=0.8, tol_lo=0.05, tol_hi=0.05)
    ctx = sipo.sipo_create(dict(nx=n, ny=n, nz=n, angles=ang, n_det=n, vial_radius=15.0), tgt, cp,
                           dict(storage=st, kkt_tol=0.0, max_iter=256))
    res = sipo.sipo_solve(ctx)
    dose = torch.empty((n, n, n), dtype=dt, device="cuda")
    lab = torch.empty((n, n, n), dtype=torch.uint8, device="cuda")
    sipo.sipo_get_array(ctx, 5, dose)
    sipo.sipo_get_array(ctx, 0, lab)
    f_t = torch.from_numpy(tgt).cuda()
    f_crit = res["f_crit"]
    lower_scale = (1.0 - cp["tol_lo"]) / f_crit if kase == 1 else 1.0 / f_crit
    torch.cuda.synchronize()
    expected = np.array([res["dtvr_f"], res["dsr"], res["psr_f"], res["alpha"], res["s"]])
    first = _abi.sipo_dose_metrics_noalloc(dose, lab, f_t, f_crit, lower_scale)
    free_before = torch.cuda.mem_get_info()[0]
    second = _abi.sipo_dose_metrics_noalloc(dose, lab, f_t, f_crit, lower_scale)
    free_after = torch.cuda.mem_get_info()[0]
    np.testing.assert_allclose(first, expected, rtol=tol)
    np.testing.assert_allclose(second, expected, rtol=tol)
    assert free_after == free_before
    sipo.sipo_destroy(ctx)


def test_noalloc_rejects_sizes_beyond_the_static_scratch(sipo):
    from paper_2604_08997_gb300 import _abi
    lib = _abi.load()
    d = torch.zeros(8, device="cuda")
    lab = torch.zeros(8, dtype=torch.uint8, device="cuda")
    f = torch.ones(8, device="cuda")
    out = (ctypes.c_double * 5)()
    rc = lib.sipo_dose_metrics_noalloc(ctypes.c_void_p(d.data_ptr()), 0, ctypes.c_void_p(lab.data_ptr()),
                                       ctypes.c_void_p(f.data_ptr()), (1 << 27) + 1, 1.0, 1.0, out, None)
    assert rc == -1
    assert b"static scratch limit" in lib.sipo_last_error()
