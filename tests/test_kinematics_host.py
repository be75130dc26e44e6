"""The device kinematics header (csrc/device/mf_kinematics.cuh) built for the
host and compared with the oracle (CPU only):

* Philox4x64-10 outputs bit for bit;
* the mass-ratio root x and its complement d = 1 - x for daughter systems of
  m = 2..6 massless particles, including r -> 0 and r -> 1 where d must keep
  full relative precision (the general-m solver is not reached by the
  processes the GPU tests run);
* flat massless momenta from the same unit numbers, including mass ratios
  1 - 1e-12 where a daughter's energy is ~1e-6 of sqrt(s-hat) and must still
  agree to rounding relative to itself.
"""
import math
import os
import shutil
import subprocess

import numpy as np
import pytest

from oracle import phasespace as ps
from oracle import philox as ph

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
EPS = np.finfo(np.float64).eps


@pytest.fixture(scope="module")
def kc(tmp_path_factory):
    gxx = shutil.which("g++")
    if gxx is None:
        pytest.skip("no host C++ compiler")
    exe = tmp_path_factory.mktemp("kc") / "kinematics_check"
    subprocess.run([gxx, "-std=c++17", "-O1", "-I", os.path.join(ROOT, "paper_2106_10279_gb300", "csrc", "device"),
                    os.path.join(ROOT, "tests", "kinematics_check.cpp"), "-o", str(exe)], check=True)

    def run(lines):
        res = subprocess.run([str(exe)], input="\n".join(lines) + "\n", capture_output=True, text=True, check=True)
        return [l.split() for l in res.stdout.strip().splitlines()]
    return run


def test_philox_bits_match_the_oracle(kc):
    rng = np.random.default_rng(5)
    cases = [(0, 0, 0, 0, 0, 0), (2 ** 64 - 1, 2 ** 64 - 1, 2 ** 64 - 1, 2 ** 64 - 1, 2 ** 64 - 1, 2 ** 64 - 1)]
    cases += [tuple(int(v) for v in rng.integers(0, 2 ** 63, 6, dtype=np.int64)) for _ in range(20)]
    out = kc(["philox " + " ".join(str(v) for v in c) for c in cases])
    for c, o in zip(cases, out):
        ref = ph.philox4x64_10(np.array([c[:4]], dtype=np.uint64), np.array(c[4:], dtype=np.uint64))
        assert [int(v) for v in o] == [int(v) for v in np.asarray(ref).ravel()]


@pytest.mark.parametrize("m", [2, 3, 4, 5, 6])
def test_mass_ratio_and_complement(kc, m):
    r = np.array([1e-14, 1e-9, 1e-3, 0.25, 0.5, 0.5000000001, 0.75, 0.999, 1 - 1e-9, 1 - 1e-12, 1 - 2 ** -52])
    out = np.array([[float(v) for v in o] for o in kc([f"ratio {m} {float(v)!r}" for v in r])])
    x, d = out[:, 0], out[:, 1]
    xo, do = ps._mass_ratio(r, m, complement=True)
    # both sides solve for the same root; each result is within a few ulps of
    # it (the oracle's bisection is exact to the last bit)
    assert np.all(np.abs(x - xo) <= 4 * np.spacing(xo))
    assert np.all(np.abs(d - do) <= 8 * EPS * do + 4 * np.spacing(do)), np.abs(d / do - 1).max()
    # d = 1 - x wherever that subtraction is exact enough to check
    lo = r <= 0.5
    assert np.all(np.abs(d[lo] - (1 - x[lo])) <= 2 * EPS)
    if m == 2:
        assert np.all(np.abs(d - np.sqrt(1 - r)) <= 2 * np.spacing(d))


@pytest.mark.parametrize("n", [2, 3, 4, 5])
def test_massless_momenta_match_the_oracle(kc, n):
    rng = np.random.default_rng(40 + n)
    N = 64
    u = rng.random((3 * n - 4, N))
    # mass ratios at both ends of their range, angles at the poles
    for k in range(n - 2):
        u[3 * k + 2, :8] = 1 - 1e-12
        u[3 * k + 2, 8:12] = 1e-12
    u[0, 12:16] = 1.0
    rs = rng.uniform(100, 13000, N)
    lines = [f"diet {n} {float(rs[i])!r} " + " ".join(repr(float(v)) for v in u[:, i]) for i in range(N)]
    got = np.array([[float(v) for v in o] for o in kc(lines)]).reshape(N, n, 4)
    ref = ps.massless_diet(u, rs)
    assert np.max(np.abs(got - ref) / rs[:, None, None]) < 1e-13
    # every energy to rounding relative to itself, even when it is ~1e-6 sqrt(s)
    e_got, e_ref = got[:, :, 0], ref[:, :, 0]
    assert np.max(np.abs(e_got - e_ref) / e_ref) < 1e-12
