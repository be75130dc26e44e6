"""Helicity sampling on the GPU (one uniformly drawn helicity per point,
scaled by the helicity count) against the oracle's restatement on the same
points and draws, and a sampled Vegas iteration against the full sum within
the combined Monte Carlo errors."""
import numpy as np
import pytest

import workloads as W
from _tolerance import fp64_tolerance, relerr

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__ as g
    g.build()
    from paper_2106_10279_gb300 import api
    return torch, api


@pytest.mark.parametrize("name,n", [("gg_ttx", 1500), ("uux_ttxg", 400), ("gg_ttxg", 500)])
def test_sampled_integrand_matches_the_oracle(env, oracle_processes, name, n):
    torch, api = env
    from oracle.integrand import Integrand
    wl = W.WORKLOADS[name]
    I = Integrand(wl, process=oracle_processes(name))
    hels = I.nonzero_helicities()
    proc = api.Process.from_workload(wl)
    assert np.array_equal(proc.helicities(), np.array(hels, dtype=np.int8))
    proc.set_helicity_sampling(True, seed=77)
    x = W.uniform_points(wl.ndim, n, 404)
    xd = torch.from_numpy(x).cuda()
    got = proc.integrand(xd, "fp64").cpu().numpy()
    ref, pick = I.sampled(x, 77, hels)
    full, tol = fp64_tolerance(I, x)
    assert np.array_equal(got == 0, ref == 0)
    # one helicity's |M_h|^2 carries the rounding of amplitudes of the size of
    # the whole sum: the bound is relative to the larger of the sampled value
    # and the full helicity sum at the point
    err = np.abs(got - ref)
    scale = np.maximum(np.abs(ref), np.abs(full))
    assert np.all(err <= tol * scale), (np.max(err / scale), int(np.argmax(err / (tol * scale))))
    mixed = proc.integrand(xd, "mixed").cpu().numpy()
    rm = relerr(mixed, ref)[ref != 0]
    assert np.median(rm) <= 1e-5
    assert np.all(np.abs(mixed - ref) <= 1e-3 * scale)      # same scale as above
    # switching it off restores the full helicity sum
    proc.set_helicity_sampling(False)
    full = proc.integrand(xd, "fp64").cpu().numpy()
    ref_full, tol_full = fp64_tolerance(I, x)
    assert np.all(relerr(full, ref_full) <= tol_full)


def test_sampled_vegas_iteration_is_consistent(env):
    torch, api = env
    wl = W.GG_TTXG
    proc = api.Process.from_workload(wl)
    g_full, g_samp = api.Vegas(wl.ndim), api.Vegas(wl.ndim)
    r_full = g_full.iterate(proc, 400_000, 5, "mixed")
    proc.set_helicity_sampling(True, seed=1)
    r_samp = g_samp.iterate(proc, 400_000, 5, "mixed")
    assert r_samp["n_nonzero"] == r_full["n_nonzero"]          # same points pass the cuts
    d = abs(r_samp["integral"] - r_full["integral"])
    assert d < 5 * np.hypot(r_samp["error"], r_full["error"])
    assert r_samp["error"] > r_full["error"]                  # sampling adds variance


@pytest.mark.parametrize("name,n", [("gg_ttx", 1500), ("uux_ttxg", 400), ("gg_ttxg", 500)])
def test_pair_sampled_integrand_matches_the_oracle(env, oracle_processes, name, n):
    # one helicity pair per point (mode 2): the library's pair table is the
    # grouping of the oracle's kept helicities at the pair leg, and f is the
    # oracle's pair-sampled estimator on the same draws
    torch, api = env
    from oracle.integrand import Integrand
    wl = W.WORKLOADS[name]
    I = Integrand(wl, process=oracle_processes(name))
    hels = [tuple(h) for h in I.nonzero_helicities()]
    proc = api.Process.from_workload(wl)
    info = proc.info
    assert info["n_pairs"] > 0
    pairs = Integrand.helicity_pairs(hels, info["pair_leg"])
    table = proc.helicity_pairs()
    rows = [tuple(h) for h in proc.helicities()]
    assert rows == hels
    assert [(rows[a] if a >= 0 else None, rows[b] if b >= 0 else None) for a, b in table] == pairs
    proc.set_helicity_sampling(2, seed=77)
    x = W.uniform_points(wl.ndim, n, 404)
    xd = torch.from_numpy(x).cuda()
    got = proc.integrand(xd, "fp64").cpu().numpy()
    ref, pick = I.sampled_pairs(x, 77, pairs)
    full, tol = fp64_tolerance(I, x)
    assert np.array_equal(got == 0, ref == 0)
    err = np.abs(got - ref)
    scale = np.maximum(np.abs(ref), np.abs(full))
    assert np.all(err <= tol * scale), (np.max(err / scale), int(np.argmax(err / (tol * scale))))
    mixed = proc.integrand(xd, "mixed").cpu().numpy()
    assert np.all(np.abs(mixed - ref) <= 1e-3 * scale)
    assert np.median(relerr(mixed, ref)[ref != 0]) <= 1e-5


def test_pair_sampled_vegas_iteration_is_consistent(env):
    torch, api = env
    wl = W.GG_TTXG
    proc = api.Process.from_workload(wl)
    g_full, g_one, g_pair = api.Vegas(wl.ndim), api.Vegas(wl.ndim), api.Vegas(wl.ndim)
    r_full = g_full.iterate(proc, 400_000, 5, "mixed")
    proc.set_helicity_sampling(1, seed=1)
    r_one = g_one.iterate(proc, 400_000, 5, "mixed")
    proc.set_helicity_sampling(2, seed=1)
    r_pair = g_pair.iterate(proc, 400_000, 5, "mixed")
    assert r_pair["n_nonzero"] == r_full["n_nonzero"]
    d = abs(r_pair["integral"] - r_full["integral"])
    assert d < 5 * np.hypot(r_pair["error"], r_full["error"])
    # a pair covers two helicities: less spread than one helicity per point
    assert r_full["error"] < r_pair["error"] < r_one["error"]
    with pytest.raises(RuntimeError):
        proc.set_helicity_sampling(3)
