"""Helicity pairs: two helicity assignments that differ only at one leg are
evaluated by one program that computes the wavefunctions not depending on
that leg once.  Checked here: the pair table against the oracle's list of
non-vanishing helicities, and the paired helicity sum against a twin process
that evaluates one helicity at a time (created with pairs switched off), in
FP64 and mixed precision, for integrands and a Vegas iteration.  The oracle
parity tests of the integrand run through the pairs as well (they are the
default wherever they save work).
"""

import numpy as np
import pytest

import workloads as W

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


def _unpaired(api, wl):
    return api.Process.from_workload(wl, options={"helicity_pairs": 0})


@pytest.mark.parametrize("name", ["gg_ttx", "uux_ttx", "gg_ttxg", "uux_ttxg", "gg_ttxgg"])
def test_pair_table_covers_the_kept_helicities(env, oracle_processes, name):
    torch, api = env
    from oracle.integrand import Integrand
    wl = W.WORKLOADS[name]
    proc = api.Process.from_workload(wl)
    info = proc.info
    hels = np.array(Integrand(wl, process=oracle_processes(name)).nonzero_helicities(), dtype=np.int8)
    assert np.array_equal(proc.helicities(), hels)
    if info["n_pairs"] == 0:
        assert info["pair_leg"] == -1
        assert info["flops_helicity_sum"] == pytest.approx(info["n_hel"] * info["flops_per_hel"], rel=1e-12)
        return
    L = info["pair_leg"]
    assert 0 <= L < wl.n_out + 2
    # the pairs are the distinct assignments of the other legs
    others = {tuple(np.delete(h, L)) for h in hels}
    assert info["n_pairs"] == len(others)
    # the helicity sum costs less than evaluating each helicity in full
    assert info["flops_helicity_sum"] < info["n_hel"] * info["flops_per_hel"]
    assert info["flops_helicity_sum"] > 0.25 * info["n_hel"] * info["flops_per_hel"]


@pytest.mark.parametrize("name,n", [("gg_ttx", 3000), ("gg_ttxg", 1500), ("uux_ttxg", 800), ("gg_ttxgg", 300)])
def test_pairs_match_one_helicity_at_a_time(env, name, n):
    torch, api = env
    wl = W.WORKLOADS[name]
    proc = api.Process.from_workload(wl)
    if proc.info["n_pairs"] == 0:
        pytest.skip("no helicity pairs for this process")
    twin = _unpaired(api, wl)
    assert twin.info["n_pairs"] == 0
    x = torch.from_numpy(W.uniform_points(wl.ndim, n, 808)).cuda()
    # FP64: the per-helicity values are the same arithmetic; only the order
    # of the helicity sum differs (pairs of the pair leg are neighbours)
    f = proc.integrand(x, "fp64").cpu().numpy()
    g = twin.integrand(x, "fp64").cpu().numpy()
    assert np.array_equal(f == 0, g == 0)
    nz = f != 0
    assert nz.sum() > 0.3 * n
    assert np.max(np.abs(f[nz] / g[nz] - 1)) <= 1e-13
    # mixed precision: the same FP32 arithmetic per helicity as well
    fm = proc.integrand(x, "mixed").cpu().numpy()
    gm = twin.integrand(x, "mixed").cpu().numpy()
    assert np.array_equal(fm == 0, gm == 0)
    assert np.max(np.abs(fm[nz] / gm[nz] - 1)) <= 1e-5
    assert np.median(np.abs(fm[nz] / gm[nz] - 1)) <= 1e-6


def test_paired_vegas_iteration_matches_unpaired(env):
    torch, api = env
    wl = W.GG_TTXG
    proc = api.Process.from_workload(wl)
    twin = _unpaired(api, wl)
    for prec, tol in (("fp64", 1e-12), ("mixed", 1e-6)):
        a, b = api.Vegas(wl.ndim), api.Vegas(wl.ndim)
        ra = a.iterate(proc, 300_000, 5, prec)
        rb = b.iterate(twin, 300_000, 5, prec)
        assert ra["n_nonzero"] == rb["n_nonzero"]
        assert abs(ra["sigma"] / rb["sigma"] - 1) <= tol, (prec, ra["sigma"], rb["sigma"])
        assert np.array_equal(a.histogram()[1], b.histogram()[1])
