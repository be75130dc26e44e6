"""The generated diagram programs built for the host in double precision and
compared with the oracle's per-helicity |M|^2 (CPU only):

* the program of one helicity, for every helicity row, which checks the code
  generator's schedule, its amplitude units (FFV amplitudes with the same
  spinors and colour coefficients equal up to +-1 or +-i evaluated once on
  the combined vector current; the default for long programs, forced on for
  all in a second pass) and the vertex routines;
* the program of a helicity pair (the two rows that differ only at the pair
  leg, evaluated with the wavefunctions independent of that leg shared), for
  every pair.

Bound: 1e-12 of the point's helicity sum per helicity, as in the GPU
per-helicity test (the same FP64 arithmetic; only the order of operations
differs from the oracle's)."""
import itertools
import os
import re
import shutil
import subprocess

import numpy as np
import pytest

import workloads as W

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


# A gauge vector for the host build: the device header's external vector
# wavefunction, with helicity code 0 returning the leg's momentum over its
# energy instead of a polarisation (a copy of the header, placed where the
# generated program looks first; the device header itself is unchanged).
_VXX_HEAD = "MF_DEV W<R> vxx(const R *k, int l, int incoming) {\n    W<R> w;\n"
_VXX_GAUGE = ("    if (l == 0) {\n        for (int m = 0; m < 4; ++m) w.c[m] = C<R>(k[m] / k[0], R(0));\n"
              "        return w;\n    }\n")


def _build(tmp, name, units, gauge=False):
    from paper_2106_10279_gb300 import api
    gxx = shutil.which("g++")
    if gxx is None:
        pytest.skip("no host C++ compiler")
    desc = api.descriptor_for_workload(W.WORKLOADS[name],
                                       options=None if units is None else {"amplitude_units": int(units)})
    src = api.mf_generate_kernel_source(desc, "fp64")
    src = src[:src.index('#include "mf_kernel.cuh"')]
    leg = int(re.search(r"constexpr int PAIR_LEG = (-?\d+);", src).group(1))
    (tmp / "mf_program_gen.h").write_text(src)
    if gauge:
        helas = open(os.path.join(ROOT, "paper_2106_10279_gb300", "csrc", "device", "mf_helas.cuh")).read()
        assert helas.count(_VXX_HEAD) == 1
        (tmp / "mf_helas.cuh").write_text(helas.replace(_VXX_HEAD, _VXX_HEAD + _VXX_GAUGE))
    exe = tmp / "program_check"
    subprocess.run([gxx, "-std=c++17", "-O1", "-w", "-I", str(tmp),
                    "-I", os.path.join(ROOT, "paper_2106_10279_gb300", "csrc", "device"),
                    os.path.join(ROOT, "tests", "program_check.cpp"), "-o", str(exe)], check=True)
    d = desc.desc
    head = [str(d.n_masses)] + [repr(float(d.masses[i])) for i in range(d.n_masses)]
    head += [str(d.n_couplings)] + [repr(float(d.couplings[i])) for i in range(2 * d.n_couplings)]

    def run(lines):
        res = subprocess.run([str(exe)], input=" ".join(head) + "\n" + "\n".join(lines) + "\n",
                             capture_output=True, text=True, check=True)
        return np.array([[float(v) for v in l.split()] for l in res.stdout.strip().splitlines()])
    return run, leg


def _line(cmd, hel, p):
    return cmd + " " + " ".join(str(int(h)) for h in hel) + " " + " ".join(repr(float(v)) for v in p.ravel())


@pytest.mark.parametrize("units", [None, "1"])
@pytest.mark.parametrize("name,n", [("ee_mumu", 4), ("gg_ttx", 6), ("uux_ttx", 6), ("gg_ttxg", 5),
                                    ("uux_ttxg", 5), ("gg_ttxgg", 3)])
def test_generated_programs_match_the_oracle(tmp_path, oracle_processes, name, n, units):
    # units None: the generator's default (amplitude units for long programs
    # only); "1": units for every program
    from oracle.integrand import Integrand
    wl = W.WORKLOADS[name]
    orc = Integrand(wl, process=oracle_processes(name))
    run, leg = _build(tmp_path, name, units)
    x = W.uniform_points(wl.ndim, 4 * n, 2024)
    p, s_hat, x1, x2, jx, w, ok = orc.kinematics(x)
    keep = ok & orc.cuts(p)
    p = p[keep][:n]
    assert p.shape[0] == n
    tot, per = orc.proc.msq_summed(p, per_helicity=True)          # [H, n], rows in table order
    nleg = p.shape[1]
    rows = list(itertools.product((-1, 1), repeat=nleg))
    assert len(rows) == per.shape[0]
    # one helicity at a time
    got = run([_line("msq", h, p[i]) for i in range(n) for h in rows]).reshape(n, len(rows))
    err = np.abs(got - per.T) / tot[:, None]
    assert err.max() <= 1e-12, (name, err.max())
    # helicity pairs: rows with the pair leg at -1, their partner at +1
    assert leg >= 0 or name == "ee_mumu"
    if leg < 0:
        return
    firsts = [h for h in rows if h[leg] == -1]
    partner = [tuple(1 if l == leg else v for l, v in enumerate(h)) for h in firsts]
    got2 = run([_line("pair", h, p[i]) for i in range(n) for h in firsts]).reshape(n, len(firsts), 2)
    ia = [rows.index(h) for h in firsts]
    ib = [rows.index(h) for h in partner]
    ea = np.abs(got2[:, :, 0] - per[ia].T) / tot[:, None]
    eb = np.abs(got2[:, :, 1] - per[ib].T) / tot[:, None]
    assert max(ea.max(), eb.max()) <= 1e-12, (name, ea.max(), eb.max())


@pytest.mark.parametrize("units", [None, "1"])
@pytest.mark.parametrize("name,n", [("gg_ttx", 4), ("gg_ttxg", 4), ("uux_ttxg", 4), ("gg_ttxgg", 2)])
def test_generated_programs_are_gauge_invariant(tmp_path, oracle_processes, name, n, units):
    # a gluon's polarisation replaced by its momentum: every amplitude of the
    # generated program (one helicity and pairs) vanishes with the other
    # gluons transverse (the Ward identity), independently of the oracle's
    # values; bound relative to the point's helicity sum, as the oracle's own
    # gauge test
    from oracle.integrand import Integrand
    wl = W.WORKLOADS[name]
    orc = Integrand(wl, process=oracle_processes(name))
    run, leg = _build(tmp_path, name, units, gauge=True)
    x = W.uniform_points(wl.ndim, 4 * n, 77)
    p, s_hat, x1, x2, jx, w, ok = orc.kinematics(x)
    p = p[ok & orc.cuts(p)][:n]
    assert p.shape[0] == n
    nleg = p.shape[1]
    rows = list(itertools.product((-1, 1), repeat=nleg))
    tot = run([_line("msq", h, p[i]) for i in range(n) for h in rows]).reshape(n, len(rows)).sum(axis=1)
    assert np.all(tot > 0)
    gluons = [l for l, lg in enumerate(wl.legs) if lg.particle == "g"]
    assert gluons
    for g in gluons:
        grow = sorted({tuple(0 if l == g else v for l, v in enumerate(h)) for h in rows})
        val = run([_line("msq", h, p[i]) for i in range(n) for h in grow]).reshape(n, len(grow))
        assert np.max(np.abs(val).sum(axis=1) / tot) < 1e-12, (name, g)
        if leg >= 0 and leg != g:
            firsts = [h for h in grow if h[leg] == -1]
            val2 = run([_line("pair", h, p[i]) for i in range(n) for h in firsts])
            assert np.max(np.abs(val2).reshape(n, -1).sum(axis=1) / tot) < 1e-12, (name, g, "pair")


def _boost(p, beta):
    """General Lorentz boost of momenta p [..., 4] by velocity beta [3]."""
    b2 = float(np.dot(beta, beta))
    gamma = 1.0 / np.sqrt(1.0 - b2)
    bp = p[..., 1:] @ beta
    out = np.empty_like(p)
    out[..., 0] = gamma * (p[..., 0] + bp)
    out[..., 1:] = p[..., 1:] + ((gamma - 1.0) * bp / b2 + gamma * p[..., 0])[..., None] * beta
    return out


@pytest.mark.parametrize("name,n", [("gg_ttx", 4), ("gg_ttxg", 4), ("uux_ttxg", 4), ("gg_ttxgg", 2)])
def test_generated_programs_are_lorentz_invariant(tmp_path, oracle_processes, name, n):
    # the helicity sum of the generated program is the same in a boosted
    # frame (denominators recomputed from the boosted momenta), independently
    # of the oracle's values
    from oracle.integrand import Integrand
    wl = W.WORKLOADS[name]
    orc = Integrand(wl, process=oracle_processes(name))
    run, leg = _build(tmp_path, name, None)
    x = W.uniform_points(wl.ndim, 4 * n, 91)
    p, s_hat, x1, x2, jx, w, ok = orc.kinematics(x)
    p = p[ok & orc.cuts(p)][:n]
    q = _boost(p, np.array([0.3, -0.45, 0.6]))
    rows = list(itertools.product((-1, 1), repeat=p.shape[1]))
    a = run([_line("msq", h, p[i]) for i in range(n) for h in rows]).reshape(n, len(rows)).sum(axis=1)
    b = run([_line("msq", h, q[i]) for i in range(n) for h in rows]).reshape(n, len(rows)).sum(axis=1)
    assert np.max(np.abs(b / a - 1)) < 1e-10, name
