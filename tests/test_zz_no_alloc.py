"""mf_vegas_iterate_static, the Vegas iteration that allocates nothing,
called through the C ABI (ctypes) and compared with mf_vegas_iterate.

Collected last so that it runs both after the other GPU tests and alone
(`pytest tests/test_zz_no_alloc.py -m gpu`): it builds everything it uses.
Two calls in a row on one grid against two mf_vegas_iterate calls on another
grid, same seed and points.  Both paths run the same compiled process
kernel, the same per-chunk accumulation and the same fixed reduction tree,
so every result is the same to the bit: estimates, errors, histograms,
counts and the refined grid compared with ==.  The device's free memory is
the same before and after a call (the first call on a device may load the
library's device code; the check is on the calls after it).
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


@pytest.mark.parametrize("name,prec,n", [("gg_ttx", 0, N), ("gg_ttxg", 1, N), ("gg_ttxgg", 3, 50_003)])
def test_static_iterations_match_vegas_iterate(env, name, prec, n):
    torch, L, api = env
    wl = W.WORKLOADS[name]
    proc = api.Process.from_workload(wl)
    pname = {0: "fp64", 1: "mixed", 3: "mixed_tc"}[prec]
    # compile the kernel first: compiling allocates, the static call does not
    proc.integrand(torch.full((wl.ndim, 8), 0.5, dtype=torch.float64, device="cuda"), pname)
    torch.cuda.synchronize()
    ref = api.Vegas(wl.ndim)
    got = api.Vegas(wl.ndim)
    for it in range(2):                                  # two calls in a row
        r_ref = ref.iterate(proc, n, 17, pname)
        torch.cuda.synchronize()
        free0 = torch.cuda.mem_get_info()[0]
        st, r = _static(L, got, proc, n, 17, prec)
        free1 = torch.cuda.mem_get_info()[0]
        assert st == L.MF_OK, L.lib().mf_last_error()
        if it > 0:
            assert free1 == free0, (free0, free1)
        for k in ("iteration", "n_events", "n_nonzero", "n_nan"):
            assert r[k] == r_ref[k], (it, k)
        for k in ("integral", "error", "sigma", "sigma_error"):
            assert r[k] == r_ref[k], (it, k, r[k], r_ref[k])
        h, c = got.histogram()
        h_ref, c_ref = ref.histogram()
        assert np.array_equal(c, c_ref)
        assert np.array_equal(h, h_ref)
        assert np.array_equal(got.grid, ref.grid)


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
