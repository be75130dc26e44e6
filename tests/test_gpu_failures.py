"""Failure detection, exercised without a GPU fault:

* an expired bounded wait: a process whose tensor-core colour sum may poll
  its MMA-completion barrier 0 times gives up every round at once; the
  kernel records the error and returns, mf_process_check reports
  MF_ETIMEOUT, the synchronous Vegas path reports it itself, and the process
  and the device stay usable;
* allocation failure: the library's allocation hook makes the n-th device
  allocation fail; mf_create_process and mf_vegas_iterate return MF_ENOMEM
  (nothing leaks into a half-built object) and succeed once the hook is
  disarmed;
* non-finite values: points with a NaN or infinite coordinate give NaN and
  raise the non-finite flag (MF_ENAN from mf_process_check); couplings so
  large that single precision overflows give non-finite Vegas weights, which
  mf_vegas_iterate counts and reports as MF_ENAN while the double-precision
  path stays finite.
"""
import ctypes as C

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
    from paper_2106_10279_gb300 import _lib as L
    from paper_2106_10279_gb300 import api
    return torch, L, api


def _x(torch, wl, n, seed):
    return torch.from_numpy(W.uniform_points(wl.ndim, n, seed)).cuda()


def test_expired_wait_is_reported_and_the_process_recovers(env):
    torch, L, api = env
    wl = W.GG_TTX
    bad = api.Process.from_workload(wl, options={"wait_polls": 0})
    good = api.Process.from_workload(wl)
    x = _x(torch, wl, 3000, 41)
    bad.integrand(x, "mixed_tc")
    torch.cuda.synchronize()
    assert L.lib().mf_process_check(bad.handle) == L.MF_ETIMEOUT
    assert b"bounded wait" in L.lib().mf_last_error()
    assert L.lib().mf_process_check(bad.handle) == L.MF_OK           # read and cleared
    # the synchronous Vegas path reports the expiry itself
    v = api.Vegas(wl.ndim)
    with pytest.raises(L.MfError) as e:
        v.iterate(bad, 20000, 3, "mixed_tc")
    assert e.value.status == L.MF_ETIMEOUT
    # the process (other precisions) and the device are still usable
    assert np.array_equal(bad.integrand(x, "mixed").cpu().numpy(), good.integrand(x, "mixed").cpu().numpy())
    f_tc = good.integrand(x, "mixed_tc").cpu().numpy()
    f64 = good.integrand(x, "fp64").cpu().numpy()
    torch.cuda.synchronize()
    assert L.lib().mf_process_check(good.handle) == L.MF_OK
    nz = f64 != 0
    assert np.median(np.abs(f_tc[nz] / f64[nz] - 1)) < 1e-5


def test_allocation_failures_return_enomem(env):
    torch, L, api = env
    wl = W.GG_TTX
    desc = api.descriptor_for_workload(wl)
    lib = L.lib()
    failed = 0
    try:
        for after in range(0, 12):
            lib.mf_debug_fail_allocation(after)
            h = C.c_void_p()
            st = lib.mf_create_process(C.byref(desc.desc), C.byref(h))
            lib.mf_debug_fail_allocation(-1)
            if st == L.MF_OK:
                lib.mf_destroy_process(h)
                break
            assert st == L.MF_ENOMEM, (after, st, lib.mf_last_error())
            assert not h.value
            failed += 1
        assert failed >= 3            # PDF rows, error flag, helicity-filter scratch at least
        # the first Vegas iteration allocates the process's point scratch
        proc = api.Process.from_workload(wl)
        v = api.Vegas(wl.ndim)
        lib.mf_debug_fail_allocation(0)
        with pytest.raises(L.MfError) as e:
            v.iterate(proc, 10000, 5, "fp64")
        assert e.value.status == L.MF_ENOMEM
    finally:
        lib.mf_debug_fail_allocation(-1)
    r = v.iterate(proc, 10000, 5, "fp64")
    ref = api.Vegas(wl.ndim).iterate(api.Process.from_workload(wl), 10000, 5, "fp64")
    assert r["integral"] == ref["integral"] and r["n_nonzero"] == ref["n_nonzero"]


def test_non_finite_points_and_weights(env):
    torch, L, api = env
    wl = W.GG_TTX
    proc = api.Process.from_workload(wl)
    x = _x(torch, wl, 2000, 43)
    clean = proc.integrand(x, "fp64").cpu().numpy()
    torch.cuda.synchronize()
    assert L.lib().mf_process_check(proc.handle) == L.MF_OK
    xb = x.clone()
    xb[0, 5] = float("nan")
    xb[2, 17] = float("inf")
    f = proc.integrand(xb, "fp64").cpu().numpy()
    torch.cuda.synchronize()
    assert np.isnan(f[5]) and np.isnan(f[17])
    keep = np.ones(f.size, bool)
    keep[[5, 17]] = False
    assert np.array_equal(f[keep], clean[keep])
    assert L.lib().mf_process_check(proc.handle) == L.MF_ENAN
    assert L.lib().mf_process_check(proc.handle) == L.MF_OK
    # |M|^2 ~ g_s^4: at alpha_s = 1e25 the colour sum of the single-precision
    # amplitudes (~1e26 each) overflows while double precision does not
    big = api.Process.from_workload(wl, alpha_s=1e25)
    r64 = api.Vegas(wl.ndim).iterate(big, 20000, 7, "fp64")
    assert r64["n_nan"] == 0 and np.isfinite(r64["integral"])
    st = L.mf_iter_result()
    v = api.Vegas(wl.ndim)
    h = (C.c_void_p * 1)(v.handle.value)
    p = (C.c_void_p * 1)(big.handle.value)
    n = (C.c_int64 * 1)(20000)
    code = L.lib().mf_vegas_iterate(h, p, n, 1, 7, L.MF_MIXED, 1, C.byref(st), None)
    assert code == L.MF_ENAN
    assert st.n_nan == r64["n_nonzero"] and st.n_events == 20000
