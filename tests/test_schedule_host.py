"""The host schedule of the probed and raced solves (sipo_schedule.h, the loop
behind sipo_solve_probe and sipo_solve_race) compiled with the host compiler
against stand-in solvers and run on the CPU: probe cadence at whole check
periods, stops at a certificate, at the rival's decision, at either cap, and
the ragged last block.  No GPU."""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_probe_and_race_schedule(tmp_path):
    cxx = shutil.which("g++") or shutil.which("c++")
    if cxx is None:
        pytest.skip("no host C++ compiler")
    exe = tmp_path / "schedule_check"
    subprocess.run([cxx, "-std=c++17", "-O1", "-Wall", "-Werror",
                    "-I", os.path.join(ROOT, "paper_2604_08997_gb300", "csrc"),
                    os.path.join(ROOT, "tests", "schedule_check.cpp"), "-o", str(exe)],
                   check=True, capture_output=True, text=True)
    out = subprocess.run([str(exe)], capture_output=True, text=True)
    assert out.returncode == 0, out.stdout + out.stderr
    assert "schedule check: ok" in out.stdout
