"""The colour sum on the tensor cores (tcgen05, split TF32) and on the CUDA
cores (FP32) through mf_colour_sum, against the FP64 colour sum of the same
amplitudes, for the colour bases of the processes (2, 4, 6 and 24 flows) with
the builder's integer colour matrices; sizes span many 128-row tiles per block
(the completion barrier's phase alternates) and a ragged last tile."""
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


@pytest.mark.parametrize("name,n", [("uux_ttx", 1000), ("uux_ttxg", 5000), ("gg_ttxg", 77_777),
                                    ("gg_ttxgg", 1000), ("gg_ttxgg", 152 * 128 * 3 + 5)])
@pytest.mark.parametrize("use_tc", [1, 0])
def test_colour_sum_matches_fp64(env, name, n, use_tc):
    torch, L, api = env
    d = api.descriptor_for_workload(W.WORKLOADS[name])
    nj = d.desc.n_jamp
    cnum = np.ctypeslib.as_array(d.desc.colour_num, shape=(nj * nj,)).astype(np.int32).copy()
    den = int(d.desc.colour_den)
    rng = np.random.default_rng(nj + n)
    scale = np.exp(rng.uniform(-3, 3, n))                   # rows of very different size
    J = (rng.standard_normal((2 * nj, n)) * scale).astype(np.float32)
    Jd = torch.from_numpy(J).cuda()
    out = torch.empty(n, dtype=torch.float32, device="cuda")
    st = L.lib().mf_colour_sum(C.c_void_p(Jd.data_ptr()), n, cnum.ctypes.data_as(C.POINTER(C.c_int32)), nj, den,
                               use_tc, C.c_void_p(out.data_ptr()), None)
    assert st == L.MF_OK, L.lib().mf_last_error()
    got = out.cpu().numpy().astype(np.float64)
    Cm = cnum.reshape(nj, nj).astype(np.float64)
    Jc = J[0::2].astype(np.float64) + 1j * J[1::2].astype(np.float64)       # [nj, n]
    ref = np.real(np.einsum("kn,kl,ln->n", Jc.conj(), Cm, Jc)) / den
    absform = np.einsum("kn,kl,ln->n", np.abs(Jc), np.abs(Cm), np.abs(Jc)) / den
    err = np.abs(got - ref) / absform
    assert err.max() < 2e-6, err.max()
    assert np.all(ref > 0)                                     # C is positive definite


@pytest.mark.parametrize("name,n", [("gg_ttx", 1500), ("uux_ttxg", 500), ("gg_ttxg", 700), ("gg_ttxgg", 300)])
def test_fused_kernel_with_tensor_core_colour_sum(env, oracle_processes, name, n):
    # MF_MIXED_TC: the integrand with the colour sum on the tensor cores, to the
    # mixed-precision bounds against the oracle and close to the FP32 path
    torch, L, api = env
    from oracle.integrand import Integrand
    from _tolerance import relerr
    wl = W.WORKLOADS[name]
    proc = api.Process.from_workload(wl)
    x = W.uniform_points(wl.ndim, n, 202)
    xd = torch.from_numpy(x).cuda()
    got = proc.integrand(xd, "mixed_tc").cpu().numpy()
    mixed = proc.integrand(xd, "mixed").cpu().numpy()
    proc.check()
    ref = Integrand(wl, process=oracle_processes(name))(x)
    assert np.array_equal(got == 0, ref == 0)
    r = relerr(got, ref)[ref != 0]
    assert np.median(r) <= 1e-5 and r.max() <= 1e-3, (np.median(r), r.max())
    r2 = relerr(got, mixed)[mixed != 0]
    assert np.median(r2) <= 1e-5, np.median(r2)


def test_vegas_iteration_with_tensor_core_colour_sum(env):
    torch, L, api = env
    wl = W.GG_TTXG
    proc = api.Process.from_workload(wl)
    a, b = api.Vegas(wl.ndim), api.Vegas(wl.ndim)
    # first iteration: same grid, same points, same cuts and bins
    ra = a.iterate(proc, 100_000, 8, "mixed_tc")
    rb = b.iterate(proc, 100_000, 8, "mixed")
    assert ra["n_nonzero"] == rb["n_nonzero"]
    assert abs(ra["sigma"] / rb["sigma"] - 1) < 1e-5
    assert np.array_equal(a.histogram()[1], b.histogram()[1])
    # second iteration on grids refined from slightly different sums
    ra = a.iterate(proc, 100_000, 8, "mixed_tc")
    rb = b.iterate(proc, 100_000, 8, "mixed")
    assert abs(ra["sigma"] / rb["sigma"] - 1) < 1e-4


@pytest.mark.parametrize("name,n", [("gg_ttx", 800), ("uux_ttx", 800), ("uux_ttxg", 300), ("gg_ttxg", 300),
                                    ("gg_ttxgg", 64)])
def test_leading_colour_matches_the_oracle(env, oracle_processes, name, n):
    # the diagonal of the colour matrix in the colour-flow (string) basis, on
    # both sides; turning it off restores the full colour sum
    torch, L, api = env
    from oracle.integrand import Integrand
    from _tolerance import fp64_tolerance, relerr
    wl = W.WORKLOADS[name]
    I = Integrand(wl, process=oracle_processes(name))
    proc = api.Process.from_workload(wl)
    x = W.uniform_points(wl.ndim, n, 505)
    xd = torch.from_numpy(x).cuda()
    proc.set_leading_colour(True)
    got = proc.integrand(xd, "fp64").cpu().numpy()
    got_mixed = proc.integrand(xd, "mixed").cpu().numpy()
    ref = I.leading_colour(x)
    full, tol = fp64_tolerance(I, x)
    assert np.array_equal(got == 0, ref == 0)
    err = np.abs(got - ref)
    scale = np.maximum(np.abs(ref), np.abs(full))
    assert np.all(err <= tol * scale), np.max(err / scale)
    rm = relerr(got_mixed, ref)[ref != 0]
    assert np.median(rm) <= 1e-5 and rm.max() <= 1e-3
    proc.set_leading_colour(False)
    back = proc.integrand(xd, "fp64").cpu().numpy()
    assert np.all(relerr(back, full) <= tol)
