"""The library's multichannel phase space against the oracle, on the CPU:

* the channels the library derives from each descriptor's program
  (mf_channels_describe) are the oracle's, key for key and in the same
  order, for every workload including gg -> tt~ggg;
* the device channel header (csrc/device/mf_channels.cuh) built for the
  host, fed the library's table (mf_channels_table), gives the oracle's
  momenta, 1/g and partition share for the same unit numbers, channel by
  channel (relative 1e-12; shares and weights of points where the oracle
  flags an empty range are not compared, there are none at these sizes);
* the same generator and share in dual numbers (the gradient kernel's
  instantiation): values and derivatives with respect to every unit number
  and m_t equal the oracle's dual numbers within the same bound;
* Neyman's allocation (mf_channels_allocate) equals the oracle's, integer
  for integer.
"""
import os
import shutil
import subprocess

import numpy as np
import pytest

import workloads as W
from oracle import channels as C
from oracle.integrand import oracle_process

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
R0 = 400.0
EPS = np.finfo(np.float64).eps


@pytest.fixture(scope="module")
def api():
    from paper_2106_10279_gb300 import api as a
    return a


@pytest.fixture(scope="module")
def cc(tmp_path_factory):
    gxx = shutil.which("g++")
    if gxx is None:
        pytest.skip("no host C++ compiler")
    exe = tmp_path_factory.mktemp("cc") / "channels_check"
    subprocess.run([gxx, "-std=c++17", "-O1", "-I", os.path.join(ROOT, "paper_2106_10279_gb300", "csrc", "device"),
                    os.path.join(ROOT, "tests", "channels_check.cpp"), "-o", str(exe)], check=True,
                   capture_output=True)

    def run(lines):
        res = subprocess.run([str(exe)], input="\n".join(lines) + "\n", capture_output=True, text=True, check=True)
        return [[float(v) for v in l.split()] for l in res.stdout.strip().splitlines()]
    return run


@pytest.mark.parametrize("name", ["ee_mumu", "gg_ttx", "uux_ttx", "gg_ttxg", "uux_ttxg", "gg_ttxgg", "gg_ttxggg"])
def test_channel_keys_match_the_oracle(api, name):
    wl = W.WORKLOADS[name]
    lib_keys = api.mf_channels_describe(api.descriptor_for_workload(wl))
    ora_keys = [c.key for c in C.derive_channels(oracle_process(wl))]
    assert lib_keys == ora_keys
    assert len(lib_keys) >= 1


def _fmt(v):
    return repr(float(v))


@pytest.mark.parametrize("name,n_ch,n_pts", [("ee_mumu", None, 40), ("gg_ttx", None, 40), ("uux_ttxg", None, 30),
                                             ("gg_ttxg", None, 20), ("gg_ttxgg", 24, 8), ("gg_ttxggg", 12, 4)])
def test_generation_and_share_match_the_oracle(api, cc, name, n_ch, n_pts):
    wl = W.WORKLOADS[name]
    table = api.mf_channels_table(api.descriptor_for_workload(wl))
    chans = C.derive_channels(oracle_process(wl))
    assert int(table[0]) == len(chans)
    fm = np.array([wl.m_top if l.particle.startswith("t") else 0.0 for l in wl.legs if not l.incoming])
    n = len(fm)
    rng = np.random.default_rng(77)
    picks = range(len(chans)) if n_ch is None else sorted(rng.choice(len(chans), n_ch, replace=False))
    lines = ["table %d %s" % (len(table), " ".join(str(int(v)) for v in table))]
    cases = []
    for i in picks:
        u = rng.random((3 * n - 4, n_pts))
        u[:, 0] = 0.5            # one central point per channel
        rs = 400.0 + 3000.0 * rng.random(n_pts)
        for e in range(n_pts):
            lines.append("gen %d %d %s %s %s %s %s %s" % (n, i, _fmt(rs[e]), _fmt(R0), _fmt(R0), _fmt(wl.m_top),
                                                           " ".join(_fmt(v) for v in fm),
                                                           " ".join(_fmt(v) for v in u[:, e])))
        cases.append((i, u, rs))
    out = iter(cc(lines))
    for i, u, rs in cases:
        p, inv_g, ok = C.generate(chans[i], u, rs, fm, R0, R0, [wl.m_top])
        pa = np.stack([rs / 2, 0 * rs, 0 * rs, rs / 2], axis=1)
        share = C.partition(chans, pa, p, R0, R0, [wl.m_top])[:, i]
        for e in range(len(rs)):
            row = next(out)
            assert int(row[0]) == int(ok[e])
            if not ok[e]:
                continue
            # a propagator factor 1/(|x - M^2| + r)^2 moves by 2 |dx| / (|x - M^2| + r) when its
            # invariant x, formed from components of size up to sqrt(s-hat), moves by
            # |dx| ~ eps s-hat: the share's condition number is at most 2 s-hat / r0 per factor;
            # the t-channel density's (M^2 + t0 - t) has the same bound
            kappa = 2.0 * rs[e] ** 2 / R0
            assert abs(row[1] / inv_g[e] - 1) <= 1e-12 + 64 * EPS * kappa, (chans[i].key, e)
            assert abs(row[2] - share[e]) <= (1e-12 + 64 * EPS * kappa) * share[e] + 1e-300, (chans[i].key, e)
            q = np.array(row[3:]).reshape(n, 4)
            assert np.max(np.abs(q - p[e])) <= 1e-12 * rs[e], (chans[i].key, e)


def test_allocation_matches_the_oracle(api):
    rng = np.random.default_rng(9)
    for _ in range(50):
        K = int(rng.integers(1, 120))
        sigma = list(rng.random(K) * 10 ** rng.uniform(-3, 3, K))
        if rng.random() < 0.2:
            sigma[int(rng.integers(K))] = 0.0
        N = int(rng.integers(K * 10, 10 ** 7))
        floor = int(rng.integers(0, N // K + 1))
        assert api.mf_channels_allocate(sigma, N, floor) == C.allocate(sigma, N, floor)
        n_prev = [int(v) for v in rng.integers(0, 5000, K)]
        m0 = float(rng.choice([0.0, 10.0, 1000.0]))
        assert api.mf_channels_allocate(sigma, N, floor, n_prev, m0) == C.allocate(sigma, N, floor, n_prev, m0)
    assert api.mf_channels_allocate([0.0] * 7, 1000, 3) == C.allocate([0.0] * 7, 1000, 3)
    from paper_2106_10279_gb300 import _lib as L
    with pytest.raises(RuntimeError):
        api.mf_channels_allocate([1.0, 1.0], 10, 8)
    with pytest.raises(RuntimeError):
        api.mf_channels_allocate([1.0, -1.0], 10, 1)
    assert L.MF_EINVAL != 0


@pytest.mark.parametrize("name,n_ch", [("gg_ttx", None), ("uux_ttxg", None), ("gg_ttxg", 6), ("gg_ttxgg", 6)])
def test_dual_generation_matches_the_oracle(api, cc, name, n_ch):
    # the device header's channel generator and share in dual numbers (as the
    # gradient kernel runs them), built for the host: values and derivatives
    # with respect to every unit number and m_t against the oracle's own
    # dual numbers through its generator and partition
    from oracle.dual import Dual
    wl = W.WORKLOADS[name]
    table = api.mf_channels_table(api.descriptor_for_workload(wl))
    chans = C.derive_channels(oracle_process(wl))
    fm = np.array([wl.m_top if l.particle.startswith("t") else 0.0 for l in wl.legs if not l.incoming])
    n = len(fm)
    K = 3 * n - 3
    rng = np.random.default_rng(19)
    picks = range(len(chans)) if n_ch is None else sorted(rng.choice(len(chans), n_ch, replace=False))
    lines = ["table %d %s" % (len(table), " ".join(str(int(v)) for v in table))]
    cases = []
    for i in picks:
        for _ in range(3):
            u = 0.05 + 0.9 * rng.random(3 * n - 4)
            rs = float(600.0 + 2400.0 * rng.random())
            lines.append("gend %d %d %s %s %s %s %s %s" % (n, i, _fmt(rs), _fmt(R0), _fmt(R0), _fmt(wl.m_top),
                                                            " ".join(_fmt(v) for v in fm),
                                                            " ".join(_fmt(v) for v in u)))
            cases.append((i, u, rs))
    out = cc(lines)
    for (i, u, rs), row in zip(cases, out):
        ud = np.zeros((3 * n - 4, 1, K))
        for j in range(3 * n - 4):
            ud[j, 0, j] = 1.0
        U = Dual(u[:, None], ud)
        mt = Dual(np.array(wl.m_top), np.eye(K)[K - 1])
        fmd = [mt if m > 0 else Dual(np.array(0.0), np.zeros(K)) for m in fm]
        rsa = np.array([rs])
        p, inv_g, ok = C.generate(chans[i], U, rsa, fmd, R0, R0, [mt])
        pa = np.stack([rsa / 2, 0 * rsa, 0 * rsa, rsa / 2], axis=1)
        share = C.partition(chans, pa, p, R0, R0, [mt])[:, i]
        assert int(row[0]) == int(ok[0])
        vals = np.array(row[1:]).reshape(-1, K + 1)
        ref = [inv_g[0], share[0]] + [p[0, a, q] for a in range(n) for q in range(4)]
        for got, r in zip(vals, ref):
            rv, rd = float(np.asarray(r.v)), np.asarray(r.d).reshape(-1)
            scale = max(abs(rv), np.abs(rd).max(), 1e-300)
            kappa = 2.0 * rs ** 2 / R0
            tol = (1e-12 + 64 * EPS * kappa) * scale
            assert abs(got[0] - rv) <= tol + 1e-12 * rs, (chans[i].key, got[0], rv)
            assert np.max(np.abs(got[1:] - rd)) <= tol + 1e-12 * rs, (chans[i].key, np.max(np.abs(got[1:] - rd)))
