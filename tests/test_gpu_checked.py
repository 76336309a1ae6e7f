"""The checked build (-DSIPO_CHECKED) on the small ragged cases (GPU).

compute-sanitizer is closed on this machine, so the library has a build of its
own whose kernels test their computed indices (projector tap columns and z
offsets, backprojector detector rows and staged-box rows, epilogue z
offsets) and the finiteness of their FP64 block sums, recording a violated
check as a bit that sipo_check_flags() returns; the checks never trap.  This
test builds libsipo_checked.so and, in a separate process that loads it, runs
the operator pair with every backprojector tile on the ragged geometries of
the operator tests (scalar, one-group and two-group z paths, vial,
attenuation, PSF) and small FP64, FP32 and BF16 solves, then asserts that no
check fired.
"""
import os
import subprocess
import sys

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)


def _exercise():
    """Runs in the child process (SIPO_LIBRARY=checked); prints the flags."""
    sys.path.insert(0, ROOT)
    sys.path.insert(0, HERE)
    import torch
    import paper_2604_08997_gb300 as sipo
    from paper_2604_08997_gb300 import _abi
    from test_gpu_operators import CASES, _ctx
    from synthetic.targets import discs_2d, uniform_angles
    assert _abi.LIB_PATH.endswith("libsipo_checked.so")
    rng = np.random.default_rng(3)
    for case in CASES:
        for st, dt in ((sipo.SIPO_F32, torch.float32), (sipo.SIPO_F64, torch.float64)):
            for tile in range(sipo.sipo_tile_count()):
                ctx, ogeo, _ = _ctx(sipo, case, st, tile=tile)
                vol = torch.tensor(rng.uniform(-1, 1, ogeo.vol_shape), dtype=dt, device="cuda")
                sino = torch.tensor(rng.uniform(-1, 1, ogeo.sino_shape), dtype=dt, device="cuda")
                sipo.sipo_project(ctx, vol, torch.empty_like(sino))
                sipo.sipo_backproject(ctx, sino, torch.empty_like(vol))
                torch.cuda.synchronize()
                sipo.sipo_destroy(ctx)
    # solves: tiny 2-D in every case, FP64; a 256-deep stack in FP32 and BF16
    t2 = discs_2d(10, n_discs=1, r_range=(2.0, 3.0), container_radius=4.0, seed=3)
    geo2 = dict(nx=10, ny=10, nz=1, angles=uniform_angles(8), n_det=15)
    for kase, extra in ((0, {}), (1, dict(tol_lo=0.1, tol_hi=0.1)), (2, dict(inhibit_ratio=0.6)),
                        (2, dict(inhibit_ratio=0.3))):
        ctx = sipo.sipo_create(geo2, t2, dict(kase=kase, band_width=2, **extra),
                               dict(storage=sipo.SIPO_F64, kkt_tol=1e-8, max_iter=4096))
        sipo.sipo_solve(ctx)
        sipo.sipo_destroy(ctx)
    n, nz = 20, 256
    tgt = np.zeros((n, n, nz), np.float32)
    tgt[6:14, 7:13, 40:200] = 1.0
    geo3 = dict(nx=n, ny=n, nz=nz, angles=uniform_angles(27), n_det=29, vial_radius=9.5, mu=0.01)
    for st in (sipo.SIPO_F32, sipo.SIPO_BF16):
        for tile in (2, 4, 5):
            ctx = sipo.sipo_create(geo3, tgt, dict(kase=2, inhibit_ratio=0.7, band_width=2),
                                   dict(storage=st, kkt_tol=0.0, max_iter=128, tile_cfg=tile))
            sipo.sipo_solve(ctx)
            sipo.sipo_destroy(ctx)
    print("CHECK_FLAGS", hex(_abi.load().sipo_check_flags()), flush=True)


def test_checked_build_records_no_violation():
    sys.path.insert(0, ROOT)
    from paper_2604_08997_gb300.build import build
    build(checked=True)
    env = dict(os.environ, SIPO_LIBRARY="checked")
    r = subprocess.run([sys.executable, os.path.abspath(__file__), "--exercise"], env=env, cwd=ROOT,
                       capture_output=True, text=True, timeout=1200)
    assert r.returncode == 0, r.stdout[-2000:] + r.stderr[-4000:]
    line = [l for l in r.stdout.splitlines() if l.startswith("CHECK_FLAGS")][-1]
    flags = int(line.split()[1], 16)
    assert flags & 0x40000000, "the child did not load the checked build"
    assert flags & 0xffff == 0, f"checks fired: {flags:#x}"


if __name__ == "__main__" and "--exercise" in sys.argv:
    _exercise()
