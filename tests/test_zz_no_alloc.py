"""mf_vegas_iterate_static, the Vegas iteration that allocates nothing,
called through the C ABI (ctypes) and compared with mf_vegas_iterate.

Collected last so that it runs both after the other GPU tests and alone
(`pytest tests/test_zz_no_alloc.py -m gpu`): it builds everything it uses.
Two calls in a row on one grid against two mf_vegas_iterate calls on another
grid, same seed and points: estimates, errors and histograms within 1e-12
relative, counts and point totals exact, grids after refinement within 1e-12.
"""
import ctypes as C

import numpy as np
import pytest

import workloads as W

pytestmark = pytest.mark.gpu

N = 200_003                  # ragged: 49 chunks, the last one partial


@pytest.fixture(scope="module")
def env():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__ as g
    g.build()
    from paper_2106_10279_gb300 import _lib as L
    from paper_2106_10279_gb300 import api
    return torch, L, api


def _static(L, grid, proc, n, seed, prec, refine=1):
    out = L.mf_iter_result()
    st = L.lib().mf_vegas_iterate_static(grid.handle, proc.handle, n, seed, prec, refine, C.byref(out), None)
    return st, {name: getattr(out, name) for name, _ in out._fields_}


def _close(a, b, rel=1e-12):
    return abs(a - b) <= rel * max(abs(a), abs(b))


@pytest.mark.parametrize("name,prec", [("gg_ttx", 0), ("gg_ttxg", 1)])
def test_static_iterations_match_vegas_iterate(env, name, prec):
    torch, L, api = env
    wl = W.WORKLOADS[name]
    proc = api.Process.from_workload(wl)
    pname = {0: "fp64", 1: "mixed"}[prec]
    # compile the kernel first: compiling allocates, the static call does not
    proc.integrand(torch.full((wl.ndim, 8), 0.5, dtype=torch.float64, device="cuda"), pname)
    torch.cuda.synchronize()
    ref = api.Vegas(wl.ndim)
    got = api.Vegas(wl.ndim)
    for it in range(2):                                  # two calls in a row
        r_ref = ref.iterate(proc, N, 17, pname)
        st, r = _static(L, got, proc, N, 17, prec)
        assert st == L.MF_OK, L.lib().mf_last_error()
        for k in ("iteration", "n_events", "n_nonzero", "n_nan"):
            assert r[k] == r_ref[k], (it, k)
        for k in ("integral", "error", "sigma", "sigma_error"):
            assert _close(r[k], r_ref[k]), (it, k, r[k], r_ref[k])
        h, c = got.histogram()
        h_ref, c_ref = ref.histogram()
        assert np.array_equal(c, c_ref)
        assert np.allclose(h, h_ref, rtol=1e-12, atol=0)
        assert np.allclose(got.grid, ref.grid, rtol=1e-12, atol=1e-15)


def test_static_rejects_what_it_cannot_hold(env):
    torch, L, api = env
    wl = W.GG_TTX
    proc = api.Process.from_workload(wl)
    g = api.Vegas(wl.ndim)
    # kernel of this precision not compiled yet
    st, _ = _static(L, g, proc, 1000, 1, 1)
    assert st == L.MF_EINVAL
    assert b"not compiled" in L.lib().mf_last_error()
    proc.integrand(torch.full((wl.ndim, 8), 0.5, dtype=torch.float64, device="cuda"), "fp64")
    torch.cuda.synchronize()
    st, _ = _static(L, g, proc, L.MF_STATIC_MAX_EVENTS + 1, 1, 0)
    assert st == L.MF_EINVAL
    assert b"MF_STATIC_MAX_EVENTS" in L.lib().mf_last_error()
    st, _ = _static(L, g, proc, 1, 1, 0)
    assert st == L.MF_EINVAL
    # the largest size it accepts works and leaves the grid usable
    st, r = _static(L, g, proc, L.MF_STATIC_MAX_EVENTS, 2, 0)
    assert st == L.MF_OK, L.lib().mf_last_error()
    assert r["n_events"] == L.MF_STATIC_MAX_EVENTS and r["n_nonzero"] > 0
    assert np.all(np.diff(g.grid, axis=1) > 0)
