"""Parity of the CUDA integrand (mf_integrand, through the C ABI) with the
oracle, element by element on the same seeded points.

Tolerances: per-event relative error <= 1e-12 in the all-FP64 path, plus
64 eps times the point's condition number computed by the oracle (PDF
interpolation near x -> 1, propagator denominators q^2 - M^2 near their
poles, the production threshold), which is O(10) for typical points; median
<= 1e-5 and max <= 1e-3 in the mixed path.  Points whose f is zero (cuts,
threshold) must be zero on both sides.  Sizes span several 128-event tiles
with a ragged tail.
"""
import numpy as np
import pytest

import workloads as W
from _tolerance import fp64_tolerance, relerr

pytestmark = pytest.mark.gpu

CASES = [("ee_mumu", 1500), ("gg_ttx", 1500), ("uux_ttx", 1000), ("gg_ttxg", 700),
         ("uux_ttxg", 500), ("gg_ttxgg", 300)]


@pytest.fixture(scope="module")
def torch_cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__ as g
    g.build()
    return torch


@pytest.fixture(scope="module")
def gpu_process(torch_cuda):
    from paper_2106_10279_gb300 import api
    cache = {}

    def get(name):
        if name not in cache:
            cache[name] = api.Process.from_workload(W.WORKLOADS[name])
        return cache[name]
    return get


@pytest.fixture(scope="module")
def oracle_integrand(oracle_processes):
    from oracle.integrand import Integrand
    cache = {}

    def get(name):
        if name not in cache:
            cache[name] = Integrand(W.WORKLOADS[name], process=oracle_processes(name))
        return cache[name]
    return get


def _eval(torch, proc, x, prec):
    xd = torch.from_numpy(np.ascontiguousarray(x)).cuda()
    f = proc.integrand(xd, prec)
    torch.cuda.synchronize()
    return f.cpu().numpy()


@pytest.mark.parametrize("name,n", CASES)
def test_fp64_parity(torch_cuda, gpu_process, oracle_integrand, name, n):
    wl = W.WORKLOADS[name]
    x = W.uniform_points(wl.ndim, n, 101)
    got = _eval(torch_cuda, gpu_process(name), x, "fp64")
    ref, tol = fp64_tolerance(oracle_integrand(name), x)
    assert np.array_equal(got == 0, ref == 0)
    assert np.count_nonzero(ref) > 0.5 * n
    r = relerr(got, ref)
    assert np.all(r <= tol), (name, r.max(), int(np.argmax(r / tol)))
    assert np.median(r) <= 1e-13


@pytest.mark.parametrize("name,n", CASES)
def test_mixed_parity(torch_cuda, gpu_process, oracle_integrand, name, n):
    wl = W.WORKLOADS[name]
    x = W.uniform_points(wl.ndim, n, 202)
    got = _eval(torch_cuda, gpu_process(name), x, "mixed")
    ref = oracle_integrand(name)(x)
    assert np.array_equal(got == 0, ref == 0)
    r = relerr(got, ref)[ref != 0]
    assert np.median(r) <= 1e-5, (name, np.median(r))
    assert r.max() <= 1e-3, (name, r.max())


@pytest.mark.parametrize("name", ["ee_mumu", "gg_ttx", "gg_ttxg", "gg_ttxgg"])
def test_edge_points(torch_cuda, gpu_process, oracle_integrand, name):
    wl = W.WORKLOADS[name]
    x = W.edge_points(wl.ndim)
    got = _eval(torch_cuda, gpu_process(name), x, "fp64")
    ref, tol = fp64_tolerance(oracle_integrand(name), x)
    assert np.all(np.isfinite(got))
    assert np.array_equal(got == 0, ref == 0)
    r = relerr(got, ref)
    assert np.all(r <= tol), (r.max(), int(np.argmax(r / tol)))


@pytest.mark.parametrize("name,n", [("ee_mumu", 200), ("gg_ttx", 300), ("uux_ttx", 200), ("gg_ttxg", 200),
                                    ("uux_ttxg", 150), ("gg_ttxgg", 40)])
def test_per_helicity_parity(torch_cuda, gpu_process, oracle_integrand, name, n):
    # colour-summed |M|^2 of every helicity row, same HELAS states on both
    # sides; compared relative to the event's helicity sum
    wl = W.WORKLOADS[name]
    proc = gpu_process(name)
    orc = oracle_integrand(name)
    x = W.uniform_points(wl.ndim, n, 303)
    xd = torch_cuda.from_numpy(x).cuda()
    got = proc.helicity_msq(xd, "fp64").cpu().numpy()
    p, s_hat, x1, x2, jx, w, ok = orc.kinematics(x)
    keep = ok & orc.cuts(p)
    tot, per = orc.proc.msq_summed(p[keep], per_helicity=True)
    g = got[:, keep]
    assert g.shape == per.shape
    err = np.abs(g - per) / tot[None, :]
    assert err.max() <= 1e-12, (name, err.max(), np.unravel_index(np.argmax(err), err.shape))
    assert np.all(got[:, ~keep] == 0)


def test_empty_single_and_ragged(torch_cuda, gpu_process, oracle_integrand):
    import ctypes as C
    from paper_2106_10279_gb300 import _lib
    proc = gpu_process("gg_ttx")
    # n = 0 is a no-op, even with NULL pointers
    assert _lib.lib().mf_integrand(proc.handle, None, 0, None, 0, None) == _lib.MF_OK
    for n in (1, 31, 127, 128, 129, 257):
        x = W.uniform_points(4, n, 7 + n)
        got = _eval(torch_cuda, proc, x, "fp64")
        ref, tol = fp64_tolerance(oracle_integrand("gg_ttx"), x)
        assert np.all(relerr(got, ref) <= tol), n


def test_bit_reproducible(torch_cuda, gpu_process):
    proc = gpu_process("gg_ttxg")
    x = W.uniform_points(7, 1000, 9)
    a = _eval(torch_cuda, proc, x, "fp64")
    b = _eval(torch_cuda, proc, x, "fp64")
    assert np.array_equal(a.view(np.int64), b.view(np.int64))


def test_helicity_filtering(torch_cuda, gpu_process, oracle_integrand):
    # the kept helicities are the oracle's non-vanishing ones, in its order:
    # massless fermions conserve helicity (e+e- -> mu+mu- keeps 4 of 16,
    # uu~ -> tt~ the rows with opposite u, u~ helicities); in gg -> tt~ the
    # rows with equal gluon and opposite top helicities vanish
    info = {name: gpu_process(name).info for name in ("ee_mumu", "uux_ttx", "gg_ttx")}
    assert (info["ee_mumu"]["n_hel"], info["ee_mumu"]["n_hel_all"]) == (4, 16)
    assert info["uux_ttx"]["n_hel_all"] == 16 and info["uux_ttx"]["n_hel"] <= 8
    assert info["gg_ttx"]["n_hel"] == 12
    for name in ("ee_mumu", "uux_ttx", "gg_ttx", "gg_ttxg", "uux_ttxg"):
        got = gpu_process(name).helicities()
        ref = np.array(oracle_integrand(name).nonzero_helicities(), dtype=np.int8)
        assert np.array_equal(got, ref), name


def test_fp64_error_budget(torch_cuda, gpu_process, oracle_integrand, capsys):
    # how the FP64 errors sit against the bare 1e-12: over every workload,
    # the share of points above it and the condition number of the worst
    # point, which must lie within its own bound
    rows, total, above = [], 0, 0
    for name, n in CASES:
        wl = W.WORKLOADS[name]
        x = W.uniform_points(wl.ndim, n, 101)
        got = _eval(torch_cuda, gpu_process(name), x, "fp64")
        ref, tol = fp64_tolerance(oracle_integrand(name), x)
        _, parts = oracle_integrand(name)(x, return_parts=True)
        nz = ref != 0
        r = relerr(got, ref)[nz]
        k = parts["condition"][nz]
        total += nz.sum()
        above += int((r > 1e-12).sum())
        i = int(np.argmax(r))
        rows.append((name, int(nz.sum()), int((r > 1e-12).sum()), float(r[i]), float(k[i]),
                     float(np.median(r))))
        assert r[i] <= tol[nz][i]
    with capsys.disabled():
        for row in rows:
            print("fp64 %-9s points %5d above 1e-12 %4d worst %.2e (condition %.3g) median %.1e" % row)
    assert above <= 0.05 * total, (above, total)
