"""The hand-written adjoints of the vertex routines (csrc/device/
mf_helas_adj.cuh) against central finite differences, compiled on the host
from the same headers the gradient kernel uses (CPU only)."""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_adjoint_routines_match_finite_differences(tmp_path):
    gxx = shutil.which("g++")
    if gxx is None:
        pytest.skip("no host C++ compiler")
    exe = tmp_path / "adjoint_check"
    subprocess.run([gxx, "-std=c++17", "-O1", "-I", os.path.join(ROOT, "paper_2106_10279_gb300", "csrc", "device"),
                    os.path.join(ROOT, "tests", "adjoint_check.cpp"), "-o", str(exe)], check=True)
    res = subprocess.run([str(exe)], capture_output=True, text=True)
    lines = dict(l.split() for l in res.stdout.strip().splitlines())
    assert len(lines) == 17, res.stdout
    assert float(lines["WORST"]) < 1e-6, res.stdout
    assert res.returncode == 0
