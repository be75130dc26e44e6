"""Weighted observable histograms on the GPU (mf_vegas_observables) against
the oracle on the same Philox points of a uniform grid: transverse momentum
and rapidity of the top and pseudorapidity of the antitop in the collider
frame.  Identical bin counts; per-bin cross sections and errors within FP64
rounding (FP64 path) or the mixed-precision bound; a range holding every
point adds up to the pass's integral estimate; repeated calls give the same
bits."""
import numpy as np
import pytest

import workloads as W

pytestmark = pytest.mark.gpu

N = 40_000
SEED = 21
OBS = [("pt", 2, 20, 0.0, 500.0), ("y", 2, 16, -4.0, 4.0), ("eta", 3, 16, -4.0, 4.0)]


@pytest.fixture(scope="module")
def env(oracle_processes):
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__ as g
    g.build()
    from paper_2106_10279_gb300 import api
    from oracle import observables as ob
    from oracle import unweight as uw
    from oracle import vegas as ov
    from oracle.integrand import Integrand
    from oracle.philox import vegas_uniforms
    wl = W.GG_TTX
    I = Integrand(wl, process=oracle_processes("gg_ttx"))
    y = vegas_uniforms(SEED, 0, 0, 0, N, wl.ndim)
    x, jac, _ = ov.vegas_map(ov.uniform_grid(wl.ndim, wl.n_bins), y)
    w = I(x) * jac
    p, s_hat, x1, x2, jx, wps, ok = I.kinematics(x)
    passing = ok & I.cuts(p)
    kinds = {"pt": ob.PT, "y": ob.RAPIDITY, "eta": ob.PSEUDORAPIDITY}
    ref = ob.histograms(uw.lab_frame(p, x1, x2), passing, w, [(kinds[k], l, nb, lo, hi) for k, l, nb, lo, hi in OBS])
    return api, wl, w, ref


def test_histograms_match_the_oracle(env):
    api, wl, w, ref = env
    proc = api.Process.from_workload(wl)
    grid = api.Vegas(wl.ndim)
    got = api.observables(grid, proc, N, SEED, OBS, precision="fp64")
    for (s, e, c), (rs, re, rc), o in zip(got, ref, OBS):
        assert np.array_equal(c, rc), o
        assert c.sum() > 0.5 * N or o[0] == "pt"
        nz = rs != 0
        assert np.all(s[~nz] == 0)
        assert np.max(np.abs(s[nz] / rs[nz] - 1)) <= 1e-10, o
        assert np.max(np.abs(e[nz] / re[nz] - 1)) <= 1e-8, o
    again = api.observables(grid, proc, N, SEED, OBS, precision="fp64")
    for a, b in zip(got, again):
        for u, v in zip(a, b):
            assert np.array_equal(u, v)


def test_mixed_precision_histograms(env):
    api, wl, w, ref = env
    proc = api.Process.from_workload(wl)
    grid = api.Vegas(wl.ndim)
    got = api.observables(grid, proc, N, SEED, OBS, precision="mixed")
    for (s, e, c), (rs, re, rc), o in zip(got, ref, OBS):
        assert np.array_equal(c, rc), o
        nz = rs != 0
        assert np.max(np.abs(s[nz] / rs[nz] - 1)) <= 1e-5, o


def test_full_range_is_the_integral_of_the_pass(env):
    api, wl, w, ref = env
    proc = api.Process.from_workload(wl)
    ((s, e, c),) = api.observables(api.Vegas(wl.ndim), proc, N, SEED, [("pt", 2, 8, 0.0, 7000.0)], precision="fp64")
    r = api.Vegas(wl.ndim).iterate(proc, N, SEED, "fp64")       # the same points: iteration 0
    assert np.sum(s) == pytest.approx(r["integral"], rel=1e-12)
    assert np.sum(s) == pytest.approx(w.mean(), rel=1e-11)
    assert c.sum() == r["n_nonzero"]


def test_rejects_bad_observables(env):
    api, wl, w, ref = env
    from paper_2106_10279_gb300 import _lib as L
    proc = api.Process.from_workload(wl)
    grid = api.Vegas(wl.ndim)
    for bad in ([("pt", 1, 10, 0.0, 1.0)],             # incoming leg
                [("pt", 2, 65, 0.0, 1.0)],             # too many bins
                [("pt", 2, 10, 1.0, 1.0)],             # empty range
                [("pt", 2, 10, 0.0, 1.0)] * 5):        # too many observables
        with pytest.raises(RuntimeError):
            api.observables(grid, proc, 1000, 1, bad, precision="fp64")
    assert L.MF_MAX_OBSERVABLES == 4


def test_histograms_of_gg_ttxgg_match_the_oracle(oracle_processes):
    # the headline process: a final gluon's pT and pseudorapidity and the
    # top's rapidity, 4000 Philox points (the cuts leave about two thirds)
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__ as g
    g.build()
    from paper_2106_10279_gb300 import api
    from oracle import observables as ob
    from oracle import unweight as uw
    from oracle import vegas as ov
    from oracle.integrand import Integrand
    from oracle.philox import vegas_uniforms
    wl = W.GG_TTXGG
    n = 4000
    obs = [("pt", 4, 20, 0.0, 400.0), ("y", 2, 16, -4.0, 4.0), ("eta", 5, 16, -5.0, 5.0)]
    I = Integrand(wl, process=oracle_processes("gg_ttxgg"))
    y = vegas_uniforms(SEED, 0, 0, 0, n, wl.ndim)
    x, jac, _ = ov.vegas_map(ov.uniform_grid(wl.ndim, wl.n_bins), y)
    w = I(x) * jac
    p, s_hat, x1, x2, jx, wps, ok = I.kinematics(x)
    passing = ok & I.cuts(p)
    kinds = {"pt": ob.PT, "y": ob.RAPIDITY, "eta": ob.PSEUDORAPIDITY}
    ref = ob.histograms(uw.lab_frame(p, x1, x2), passing, w, [(kinds[k], l, nb, lo, hi) for k, l, nb, lo, hi in obs])
    proc = api.Process.from_workload(wl)
    for prec, tol in (("fp64", 1e-10), ("mixed", 1e-5)):
        got = api.observables(api.Vegas(wl.ndim), proc, n, SEED, obs, precision=prec)
        for (s, e, c), (rs, re, rc), o in zip(got, ref, obs):
            assert np.array_equal(c, rc), (prec, o)
            nz = rs != 0
            assert np.all(s[~nz] == 0)
            assert np.max(np.abs(s[nz] / rs[nz] - 1)) <= tol, (prec, o)
