"""Colour sampling (mf_process_set_colour_sampling) against the oracle.

One colour flow k per point, drawn from Philox block 12, replaces each
helicity's colour sum by NJAMP Re(conj(J_k) (C J)_k) / den.  Per point the
GPU estimate equals the oracle's estimate for the same k (same draw), with
the FP64 bound relative to the scale of the full colour sum (a single flow's
term may cancel to near zero); in mixed precision within 1e-5 (median) and
1e-3 (max) of that scale.  With the leading-colour approximation the same
holds for NJAMP C_kk |J_k|^2 / den.  Over a Vegas iteration the sampled
estimate of sigma agrees with the full colour sum within the errors.
"""
import numpy as np
import pytest

import workloads as W
from _tolerance import fp64_tolerance

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


@pytest.mark.parametrize("name,n", [("gg_ttx", 1200), ("uux_ttxg", 400), ("gg_ttxg", 400), ("gg_ttxgg", 48)])
@pytest.mark.parametrize("leading", [False, True])
def test_colour_sampled_points_match_the_oracle(env, oracle_processes, name, n, leading):
    torch, api = env
    from oracle.integrand import Integrand
    wl = W.WORKLOADS[name]
    I = Integrand(wl, process=oracle_processes(name))
    x = W.uniform_points(wl.ndim, n, 808)
    xd = torch.from_numpy(x).cuda()
    proc = api.Process.from_workload(wl)
    if leading:
        proc.set_leading_colour(True)
    proc.set_helicity_sampling(False, seed=31)        # the key of the draws on given points
    proc.set_colour_sampling(True)
    got = proc.integrand(xd, "fp64").cpu().numpy()
    got_mixed = proc.integrand(xd, "mixed").cpu().numpy()
    ref, pick = I.sampled_colour(x, 31, leading=leading)
    full, tol = fp64_tolerance(I, x)
    scale = np.abs(full) + np.abs(ref)
    assert np.array_equal(got == 0, full == 0)
    nz = full != 0
    assert np.all(np.abs(got - ref)[nz] <= (tol * scale)[nz])
    rm = (np.abs(got_mixed - ref) / scale)[nz]
    assert np.median(rm) <= 1e-5 and rm.max() <= 1e-3
    # every flow is drawn
    assert len(set(pick[nz].tolist())) == I.proc.string_basis().shape[1] or nz.sum() < 100
    proc.set_colour_sampling(False)
    back = proc.integrand(xd, "fp64").cpu().numpy()
    if not leading:
        assert np.all(np.abs(back - full)[nz] <= (tol * np.abs(full))[nz])


@pytest.mark.parametrize("name", ["gg_ttxg", "gg_ttxgg"])
def test_colour_sampled_vegas_sigma_is_unbiased(env, name):
    torch, api = env
    wl = W.WORKLOADS[name]
    n = 2_000_000 if name == "gg_ttxg" else 400_000
    proc = api.Process.from_workload(wl)
    full = api.Vegas(wl.ndim).iterate(proc, n, 5, "mixed", refine=False)
    proc.set_colour_sampling(True)
    for hs in (0, 2):
        proc.set_helicity_sampling(hs)
        r = api.Vegas(wl.ndim).iterate(proc, n, 5, "mixed", refine=False)
        assert r["n_nonzero"] == full["n_nonzero"]
        err = np.hypot(r["error"], full["error"])
        assert abs(r["integral"] - full["integral"]) < 5 * err, (hs, r, full)
        assert r["error"] >= full["error"]
    proc.set_colour_sampling(False)
    proc.set_helicity_sampling(False)
