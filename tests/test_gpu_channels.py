"""The multichannel phase space on the GPU against the oracle.

* Per point, through every channel (gg -> tt~, uu~ -> tt~g, gg -> tt~g) or a
  seeded sample of them (gg -> tt~gg): f of mf_channel_integrand in FP64
  within 1e-12 plus 64 eps times the oracle's condition number (which adds
  the bound on the channel weight's), in mixed precision within 1e-5
  (median) and 1e-3 (max); identical zero patterns.
* The first iteration of mf_vegas_iterate_channels from uniform grids draws
  the same Philox numbers as the oracle's Vegas with subprocess k for
  channel k: identical per-bin counts, integrals within 1e-11, per-bin sums
  of w^2 within the per-point FP64 tolerances (2 tol w^2 summed over the
  bin's points, plus 1e-12).
* The channels' summed cross section of gg -> tt~ agrees with the quadrature
  value and that of gg -> tt~gg with the flat phase space's, within the
  combined errors; the multichannel error is the smaller at equal points.
* The largest weight of each channel's points (mf_process_channel_max_weights)
  is the oracle's within the per-point tolerance.
* Unweighted events of a channel (mf_vegas_unweight_channel): the same
  points kept as by the oracle on the channel's Philox stream, with the same
  event weights, momentum fractions, collider-frame momenta (FP64) and
  leading-colour flows.
* Argument checks: a channel out of range, a grid count other than the
  process's channels.
"""
import math

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


def _oracle(name):
    from oracle.integrand import Integrand
    I = Integrand(W.WORKLOADS[name])
    r = (4.0 * max(W.WORKLOADS[name].pt_min_gluon, 1.0)) ** 2  # the library's default regulators
    I.use_channels(r, r)
    return I


@pytest.mark.parametrize("name,n_ch,n_pts", [("ee_mumu", None, 64), ("gg_ttx", None, 300), ("uux_ttxg", None, 200),
                                             ("gg_ttxg", None, 60), ("gg_ttxgg", 10, 12)])
def test_channel_points_match_the_oracle(env, name, n_ch, n_pts):
    torch, api = env
    wl = W.WORKLOADS[name]
    proc = api.Process.from_workload(wl)
    I = _oracle(name)
    K = proc.n_channels
    assert K == len(I.channels)
    rng = np.random.default_rng(31)
    picks = range(K) if n_ch is None else sorted(rng.choice(K, n_ch, replace=False))
    n_nonzero = 0
    for i in picks:
        x = W.uniform_points(wl.ndim, n_pts, 1000 + int(i))
        xd = torch.from_numpy(x).cuda()
        f64 = proc.channel_integrand(xd, int(i), "fp64").cpu().numpy()
        fmx = proc.channel_integrand(xd, int(i), "mixed").cpu().numpy()
        ref, tol = fp64_tolerance(lambda y, return_parts=False: I(y, return_parts=return_parts, channel=int(i)), x)
        assert np.array_equal(f64 == 0, ref == 0), i
        assert np.array_equal(fmx == 0, ref == 0), i
        assert np.all(relerr(f64, ref) <= tol), (i, np.max(relerr(f64, ref) / tol))
        nz = ref != 0
        n_nonzero += int(nz.sum())
        if nz.any():
            r = relerr(fmx, ref)[nz]
            assert np.median(r) <= 1e-5 and r.max() <= 1e-3, (i, np.median(r), r.max())
    assert n_nonzero >= 10


def _oracle_channel_iteration(I, ch, ndim, n, seed, chunk=20000):
    """The oracle's first iteration of channel ch, with a bound per bin on
    the difference of a correct FP64 evaluation: sum over the bin's points of
    2 tol w^2 (tol: the per-point FP64 tolerance)."""
    from oracle import vegas
    from oracle.philox import vegas_uniforms
    grid = vegas.uniform_grid(ndim, 50)
    s1 = s2 = 0.0
    dsum = np.zeros((ndim, 50))
    bound = np.zeros((ndim, 50))
    cnt = np.zeros_like(dsum, dtype=np.int64)
    wmax, wtol = 0.0, 0.0
    for start in range(0, n, chunk):
        m = min(chunk, n - start)
        y = vegas_uniforms(seed, 0, ch, start, m, ndim)
        x, jac, bins = vegas.vegas_map(grid, y)
        f, tol = fp64_tolerance(lambda z, return_parts=False: I(z, return_parts=return_parts, channel=ch), x)
        w = f * jac
        a, b, dd, cc = vegas.accumulate(w, bins, 50)
        s1 += a; s2 += b; dsum += dd; cnt += cc
        t2 = np.where(np.isfinite(tol), 2 * tol, 0.0) * w * w
        for j in range(ndim):
            np.add.at(bound[j], bins[j], t2)
        a = np.abs(w)
        if a.max() > wmax:
            wmax, wtol = float(a.max()), float(tol[np.argmax(a)])
    I_k, err = vegas.iteration_result(s1, s2, n)
    return I_k, err, dsum, cnt, bound, (wmax, wtol)


@pytest.mark.parametrize("name,n", [("gg_ttx", 20000), ("gg_ttxg", 3000)])
def test_first_channel_iteration_matches_the_oracle(env, name, n):
    torch, api = env
    wl = W.WORKLOADS[name]
    proc = api.Process.from_workload(wl)
    K = proc.n_channels
    grids = [api.Vegas(wl.ndim, 50, 1.5) for _ in range(K)]
    res = api.mf_vegas_iterate_channels([g.handle for g in grids], proc.handle, [n] * K, 777, "fp64")
    I = _oracle(name)
    mw = api.channel_max_weights(proc, [n] * K)
    for k in range(K):
        I_k, err, dsum, cnt, bound, (wmax, wtol) = _oracle_channel_iteration(I, k, wl.ndim, n, 777)
        assert abs(mw[k] - wmax) <= wtol * wmax, (k, mw[k], wmax)
        hs, hc = grids[k].histogram()
        assert np.array_equal(hc, cnt), k
        assert abs(res[k]["integral"] - I_k) <= 1e-11 * abs(I_k) + 1e-300, k
        assert abs(res[k]["error"] - err) <= 1e-9 * err + 1e-300, k
        assert np.all(np.abs(hs - dsum) <= bound + 1e-12 * dsum), (k, np.max(np.abs(hs - dsum) / (bound + 1e-300)))


def test_gg_ttx_sigma_by_channels(env):
    torch, api = env
    wl = W.WORKLOADS["gg_ttx"]
    proc = api.Process.from_workload(wl)
    mc = api.MultiChannel(proc)
    for it in range(6):
        r = mc.iterate(600_000, seed=2024, precision="fp64")
    assert abs(r["sigma"] - 699.76413) < 4 * r["sigma_error"], r
    assert r["sigma_error"] < 2e-3 * r["sigma"]
    mc.close()


def test_gg_ttxgg_channels_agree_with_flat_and_beat_it(env, capsys):
    torch, api = env
    wl = W.WORKLOADS["gg_ttxgg"]
    proc = api.Process.from_workload(wl)
    n = 2_000_000
    flat = api.Vegas(wl.ndim)
    for it in range(5):
        rf = flat.iterate(proc, n, seed=99, precision="mixed")
    mc = api.MultiChannel(proc)
    for it in range(5):
        rm = mc.iterate(n, seed=99, precision="mixed")
    d = abs(rf["sigma"] - rm["sigma"])
    comb = math.hypot(rf["sigma_error"], rm["sigma_error"])
    with capsys.disabled():
        print(f"gg->tt~gg: flat {rf['sigma']:.5g} +- {rf['sigma_error']:.3g}, "
              f"{proc.n_channels} channels {rm['sigma']:.5g} +- {rm['sigma_error']:.3g} pb "
              f"(last iteration: flat {rf['error']:.3g}, channels {rm['error']:.3g})")
    assert d < 4 * comb
    assert rm["error"] < rf["error"]
    mc.close()


def test_channel_argument_checks(env):
    torch, api = env
    from paper_2106_10279_gb300 import _lib as L
    wl = W.WORKLOADS["gg_ttx"]
    proc = api.Process.from_workload(wl)
    assert proc.n_channels == 3
    x = torch.from_numpy(W.uniform_points(wl.ndim, 8, 1)).cuda()
    for bad in (-1, 3):
        with pytest.raises(L.MfError) as e:
            proc.channel_integrand(x, bad)
        assert e.value.status == L.MF_EINVAL
    grids = [api.Vegas(wl.ndim) for _ in range(2)]
    with pytest.raises(L.MfError) as e:
        api.mf_vegas_iterate_channels([g.handle for g in grids], proc.handle, [100, 100], 1, "fp64")
    assert e.value.status == L.MF_EINVAL
    with pytest.raises(L.MfError) as e:
        proc.set_channel_regulators(0.0, 1.0)
    assert e.value.status == L.MF_EINVAL
    ee = api.Process.from_workload(W.WORKLOADS["ee_mumu"])
    assert ee.n_channels == 1


def test_channel_unweighting_matches_the_oracle(env):
    torch, api = env
    from oracle import unweight as uw
    from oracle import vegas as ov
    from oracle.philox import vegas_uniforms
    name, k, n, seed = "gg_ttxg", 6, 20000, 21
    wl = W.WORKLOADS[name]
    I = _oracle(name)
    op = I.proc
    y = vegas_uniforms(seed, 0, k, 0, n, wl.ndim)
    x, jac, _ = ov.vegas_map(ov.uniform_grid(wl.ndim, wl.n_bins), y)
    w = I(x, channel=k) * jac
    w_max = float(np.quantile(np.abs(w[w != 0]), 0.6))
    u = uw.accept_uniforms(seed, 0, k, n)
    keep = uw.keep(w, u, w_max)
    assert not (np.abs(np.abs(w) - u * w_max) <= 1e-9 * w_max).any()
    idx = np.nonzero(keep)[0]
    p, s_hat, x1, x2, jx, wps, ok = I.kinematics(x[:, idx], channel=k)
    p_lab = uw.lab_frame(p, x1, x2)
    pick, gap = uw.draw_flows(op.leading_colour_weights(p), uw.colour_uniforms(seed, 0, k, idx))
    proc = api.Process.from_workload(wl)
    grid = api.Vegas(wl.ndim)
    nacc, rec = api.unweight_channel(grid, proc, k, n, seed, w_max, precision="fp64")
    assert nacc == len(idx) and nacc > 100
    assert np.allclose(rec[:, 0], uw.event_weights(w[idx], w_max, n), rtol=1e-11, atol=0)
    assert np.allclose(rec[:, 1], x1, rtol=1e-13, atol=0)
    assert np.allclose(rec[:, 2], x2, rtol=1e-13, atol=0)
    mom = rec[:, 4:].reshape(nacc, len(wl.legs), 4)
    assert np.max(np.abs(mom - p_lab)) < 1e-9 * wl.sqrt_s
    clear = gap > 1e-9
    assert clear.mean() > 0.99
    assert np.array_equal(rec[clear, 3].astype(int), pick[clear])


def test_channel_histograms_match_the_oracle(env):
    # observables of one channel's pass: the points of its own stream, its
    # momenta and weights (gg -> tt~, the t-channel map)
    torch, api = env
    from oracle import observables as ob
    from oracle import unweight as uw
    from oracle import vegas as ov
    from oracle.philox import vegas_uniforms
    name, k, n, seed = "gg_ttx", 1, 30000, 5
    obs = [("pt", 2, 20, 0.0, 500.0), ("y", 2, 16, -4.0, 4.0)]
    wl = W.WORKLOADS[name]
    I = _oracle(name)
    y = vegas_uniforms(seed, 0, k, 0, n, wl.ndim)
    x, jac, _ = ov.vegas_map(ov.uniform_grid(wl.ndim, wl.n_bins), y)
    w = I(x, channel=k) * jac
    p, s_hat, x1, x2, jx, wps, ok = I.kinematics(x, channel=k)
    passing = ok & I.cuts(p)
    kinds = {"pt": ob.PT, "y": ob.RAPIDITY}
    ref = ob.histograms(uw.lab_frame(p, x1, x2), passing, w, [(kinds[a], l, nb, lo, hi) for a, l, nb, lo, hi in obs])
    proc = api.Process.from_workload(wl)
    got = api.observables(api.Vegas(wl.ndim), proc, n, seed, obs, precision="fp64", channel=k)
    for (s, e, c), (rs, re, rc), o in zip(got, ref, obs):
        assert np.array_equal(c, rc), o
        nz = rs != 0
        assert np.all(s[~nz] == 0)
        assert np.max(np.abs(s[nz] / rs[nz] - 1)) <= 1e-10, o
        assert np.max(np.abs(e[nz] / re[nz] - 1)) <= 1e-8, o


def test_multichannel_checkpoint_resumes_bit_for_bit(env):
    torch, api = env
    wl = W.WORKLOADS["gg_ttxg"]
    proc = api.Process.from_workload(wl)
    a = api.MultiChannel(proc)
    for it in range(2):
        a.iterate(100_000, seed=3, precision="fp64")
    blob = a.save()
    b = api.MultiChannel(proc)
    b.load(blob)
    assert b.sigma == a.sigma
    ra = a.iterate(100_000, seed=3, precision="fp64")
    rb = b.iterate(100_000, seed=3, precision="fp64")
    assert ra["allocation"] == rb["allocation"]
    assert (ra["integral"], ra["error"], ra["sigma"], ra["sigma_error"]) == \
        (rb["integral"], rb["error"], rb["sigma"], rb["sigma_error"])
    with pytest.raises(ValueError):
        api.MultiChannel(api.Process.from_workload(W.WORKLOADS["gg_ttx"])).load(blob)


def test_helicity_sampled_channel_iteration_matches_the_oracle(env):
    # one launch over every channel with one sampled helicity per point: point
    # i of channel k draws its helicity from Philox counter (i, 0, k, 14)
    torch, api = env
    from oracle import vegas
    from oracle.philox import philox4x64_10, to_unit, vegas_uniforms
    name, n, seed = "gg_ttxg", 1500, 4321
    wl = W.WORKLOADS[name]
    I = _oracle(name)
    hels = I.nonzero_helicities()
    proc = api.Process.from_workload(wl)
    proc.set_helicity_sampling(True, seed=9)
    K = proc.n_channels
    grids = [api.Vegas(wl.ndim, 50, 1.5) for _ in range(K)]
    res = api.mf_vegas_iterate_channels([g.handle for g in grids], proc.handle, [n] * K, seed, "fp64")
    grid = vegas.uniform_grid(wl.ndim, 50)
    for k in (0, 4, 9, K - 1):
        y = vegas_uniforms(seed, 0, k, 0, n, wl.ndim)
        x, jac, bins = vegas.vegas_map(grid, y)
        ctr = np.zeros((n, 4), dtype=np.uint64)
        ctr[:, 0] = np.arange(n, dtype=np.uint64)
        ctr[:, 2] = np.uint64(k)
        ctr[:, 3] = np.uint64(14)
        u = to_unit(philox4x64_10(ctr, np.array([seed, 0], dtype=np.uint64))[:, 0])
        pick = np.minimum((u * len(hels)).astype(np.int64), len(hels) - 1)
        f, _ = I.sampled(x, seed, hels, pick=pick, channel=k)
        w = f * jac
        s1, s2, dsum, cnt = vegas.accumulate(w, bins, 50)
        I_k, err = vegas.iteration_result(s1, s2, n)
        hs, hc = grids[k].histogram()
        assert np.array_equal(hc, cnt), k
        assert abs(res[k]["integral"] - I_k) <= 1e-10 * abs(I_k) + 1e-300, (k, res[k]["integral"], I_k)


def test_regulators_set_per_process(env):
    # other regulators than the default: the library's points and weights
    # follow the oracle's with the same s0 and t0
    torch, api = env
    from oracle.integrand import Integrand
    wl = W.WORKLOADS["gg_ttxg"]
    proc = api.Process.from_workload(wl)
    proc.set_channel_regulators(900.0, 2500.0)
    I = Integrand(wl)
    I.use_channels(900.0, 2500.0)
    x = W.uniform_points(wl.ndim, 40, 77)
    xd = torch.from_numpy(x).cuda()
    got = {}
    for ch in (0, 7, 14):
        f = proc.channel_integrand(xd, ch, "fp64").cpu().numpy()
        ref, tol = fp64_tolerance(lambda y, return_parts=False: I(y, return_parts=return_parts, channel=ch), x)
        assert np.array_equal(f == 0, ref == 0), ch
        assert np.all(relerr(f, ref) <= tol), ch
        got[ch] = f
    # and they change the weights
    proc.set_channel_regulators(6400.0, 6400.0)
    g = proc.channel_integrand(xd, 7, "fp64").cpu().numpy()
    nz = (g != 0) & (got[7] != 0)
    assert nz.sum() > 10 and np.max(np.abs(g[nz] / got[7][nz] - 1)) > 1e-3


def test_channel_iteration_with_tensor_core_sum_and_colour_sampling(env):
    # the one launch over every channel in the other kernels of a process:
    # the tensor-core colour sum (same points, integrals within the mixed
    # precision bound) and the colour-sampled kernel (an unbiased estimator
    # of the same cross section)
    torch, api = env
    wl = W.WORKLOADS["gg_ttxgg"]
    proc = api.Process.from_workload(wl)
    K = proc.n_channels
    n = [3000] * K
    ga = [api.Vegas(wl.ndim) for _ in range(K)]
    gb = [api.Vegas(wl.ndim) for _ in range(K)]
    ra = api.mf_vegas_iterate_channels([g.handle for g in ga], proc.handle, n, 11, "mixed", False)
    rb = api.mf_vegas_iterate_channels([g.handle for g in gb], proc.handle, n, 11, "mixed_tc", False)
    for k in range(K):
        assert ra[k]["n_nonzero"] == rb[k]["n_nonzero"], k
        assert abs(rb[k]["integral"] - ra[k]["integral"]) <= 1e-4 * abs(ra[k]["integral"]) + 1e-300, k
    proc.set_colour_sampling(True)
    gc = [api.Vegas(wl.ndim) for _ in range(K)]
    rc = api.mf_vegas_iterate_channels([g.handle for g in gc], proc.handle, n, 11, "mixed", False)
    proc.set_colour_sampling(False)
    sa = sum(r["integral"] for r in ra)
    sc = sum(r["integral"] for r in rc)
    ea = math.sqrt(sum(r["error"] ** 2 for r in ra))
    ec = math.sqrt(sum(r["error"] ** 2 for r in rc))
    assert all(rc[k]["n_nonzero"] == ra[k]["n_nonzero"] for k in range(K))
    assert abs(sc - sa) < 5 * math.hypot(ea, ec), (sa, ea, sc, ec)


@pytest.mark.parametrize("name,chans,n", [("gg_ttx", (0, 1, 2), 16), ("gg_ttxg", (0, 6, 14), 8)])
def test_channel_gradient_matches_the_oracle(env, name, chans, n):
    # mf_grad_channel: forward tangents through the channel's map, density
    # and partition, against the oracle's dual numbers through the same
    torch, api = env
    wl = W.WORKLOADS[name]
    proc = api.Process.from_workload(wl)
    I = _oracle(name)
    k = proc.desc.prog.alpha_s_power
    x = np.clip(W.uniform_points(wl.ndim, n, 57), 1e-3, 1 - 1e-3)
    xd = torch.from_numpy(x).cuda()
    n_nz = 0
    for ch in chans:
        f, dp, dx = (t.cpu().numpy() for t in proc.grad(xd, channel=ch))
        fo, dxo, dmo = I.gradient(x, channel=ch)
        ref, tol = fp64_tolerance(lambda y, return_parts=False: I(y, return_parts=return_parts, channel=ch), x)
        assert np.array_equal(f == 0, fo == 0), ch
        assert np.all(relerr(f, ref) <= tol), ch
        nz = fo != 0
        n_nz += int(nz.sum())
        if not nz.any():
            continue
        err = np.abs(dx - dxo)[:, nz] / (np.abs(dxo) + np.abs(fo))[:, nz]
        assert err.max() < 1e-8, (ch, err.max())
        errm = np.abs(dp[0] - dmo)[nz] / (np.abs(dmo) + np.abs(fo) / wl.m_top)[nz]
        assert errm.max() < 1e-8, (ch, errm.max())
        assert np.allclose(dp[1][nz], k * f[nz] / wl.alpha_s, rtol=1e-14)
    assert n_nz >= n
