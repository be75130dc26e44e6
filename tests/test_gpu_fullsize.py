"""Parity at the benchmark's sizes, in the launch configuration bench.py
times: one Vegas iteration of 4e7 gg->tt~gg points in mixed precision (the
timed step) and of 2e6 points in FP64 (the FP64 leg), checked on points
spread over the whole iteration that the oracle recomputes one by one from
their Philox counters: the same zeros, mixed-precision weights within the
mixed bounds, FP64 weights within the FP64 bound; and the accumulators'
point count."""
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


def _oracle_weights(I, wl, seed, idx):
    from oracle import vegas as ov
    from oracle.philox import vegas_uniforms
    grid = ov.uniform_grid(wl.ndim, wl.n_bins)
    y = np.concatenate([vegas_uniforms(seed, 0, 0, int(i), 1, wl.ndim) for i in idx], axis=1)
    x, jac, _ = ov.vegas_map(grid, y)
    f, parts = I(x, return_parts=True)
    with np.errstate(invalid="ignore"):
        tol = 1e-12 + 64 * np.finfo(float).eps * parts["condition"]
    return f * jac, np.where(np.isnan(tol), np.inf, tol)


@pytest.mark.parametrize("prec,n", [("mixed", 40_000_000), ("fp64", 2_000_000)])
def test_full_size_iteration_on_sampled_points(env, oracle_processes, prec, n):
    torch, api = env
    from oracle.integrand import Integrand
    wl = W.GG_TTXGG
    proc = api.Process.from_workload(wl)
    v = api.Vegas(wl.ndim, wl.n_bins, wl.alpha_vegas)
    seed = 1000
    r = v.iterate(proc, n, seed, prec)
    assert r["n_events"] == n and 0 < r["n_nonzero"] < n
    _, counts = v.histogram()
    assert np.all(counts.sum(axis=1) == n)
    rng = np.random.default_rng(5)
    idx = np.unique(np.concatenate([[0, n - 1], rng.integers(0, n, 62)]))
    got = api.read_weights(proc, idx)
    ref, tol = _oracle_weights(Integrand(wl, process=oracle_processes("gg_ttxgg")), wl, seed, idx)
    assert np.array_equal(got == 0, ref == 0)
    nz = ref != 0
    rel = np.abs(got[nz] - ref[nz]) / np.abs(ref[nz])
    if prec == "fp64":
        assert np.all(rel <= tol[nz]), rel.max()
    else:
        assert np.median(rel) <= 1e-5 and rel.max() <= 1e-3, (np.median(rel), rel.max())
