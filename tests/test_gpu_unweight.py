"""Unweighted events on the GPU (mf_vegas_unweight, the LHE writer) against
the oracle on the same Philox points of a uniform grid: the same points are
kept (decisions are compared away from rounding ties), with the same event
weights, momentum fractions and collider-frame momenta and the same colour
flow drawn per event (in FP64; compared away from ties of the draw); the
file holds every kept event with its flow's colour tags; the maximum weight
of a Vegas pass is the oracle's maximum."""
import numpy as np
import pytest

import workloads as W

pytestmark = pytest.mark.gpu

N = 40_000
SEED = 21


@pytest.fixture(scope="module")
def env(oracle_processes):
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__ as g
    g.build()
    from paper_2106_10279_gb300 import api
    from oracle import unweight as uw
    from oracle import vegas as ov
    from oracle.integrand import Integrand
    from oracle.philox import vegas_uniforms
    wl = W.GG_TTX
    I = Integrand(wl, process=oracle_processes("gg_ttx"))
    y = vegas_uniforms(SEED, 0, 0, 0, N, wl.ndim)
    x, jac, _ = ov.vegas_map(ov.uniform_grid(wl.ndim, wl.n_bins), y)
    w = I(x) * jac
    p, s_hat, x1, x2, jx, wps, ok = I.kinematics(x)
    return torch, api, wl, I, w, uw.lab_frame(p, x1, x2), x1, x2


def test_kept_events_match_the_oracle(env, tmp_path):
    torch, api, wl, I, w, p_lab, x1, x2 = env
    from oracle import unweight as uw
    proc = api.Process.from_workload(wl)
    grid = api.Vegas(wl.ndim)
    w_max = float(np.quantile(w[w > 0], 0.9))              # about a tenth of the points overweight
    u = uw.accept_uniforms(SEED, 0, 0, N)
    keep = uw.keep(w, u, w_max)
    tie = np.abs(np.abs(w) - u * w_max) <= 1e-9 * w_max
    assert not tie.any()
    lhe = api.LheWriter(tmp_path / "gg_ttx.lhe", [21, 21, 6, -6], [0.0, 0.0, 173.0, 173.0], xsec=700.0,
                        w_max=w_max)
    nacc, rec = api.unweight(grid, proc, N, SEED, w_max, precision="fp64", lhe=lhe)
    assert lhe.close() == nacc
    assert nacc == int(keep.sum()) and nacc > 100
    k = np.nonzero(keep)[0]
    ew = uw.event_weights(w[k], w_max, N)
    assert np.allclose(rec[:, 0], ew, rtol=1e-11, atol=0)
    assert np.allclose(rec[:, 1], x1[k], rtol=1e-13, atol=0)
    assert np.allclose(rec[:, 2], x2[k], rtol=1e-13, atol=0)
    mom = rec[:, 4:].reshape(nacc, 4, 4)
    assert np.max(np.abs(mom - p_lab[k])) < 1e-9 * 13000.0
    # the events' weights add up to the integral estimate within its spread
    est, ref = rec[:, 0].sum(), w.mean()
    assert abs(est - ref) < 5 * np.sqrt(np.sum(rec[:, 0] ** 2))
    text = open(tmp_path / "gg_ttx.lhe").read()
    assert text.count("<event>") == nacc


def test_mixed_precision_keeps_nearly_the_same_events(env):
    torch, api, wl, I, w, p_lab, x1, x2 = env
    proc = api.Process.from_workload(wl)
    grid = api.Vegas(wl.ndim)
    w_max = float(np.quantile(w[w > 0], 0.9))
    n64, _ = api.unweight(grid, proc, N, SEED, w_max, precision="fp64", capacity=0)
    nmx, _ = api.unweight(grid, proc, N, SEED, w_max, precision="mixed", capacity=0)
    assert abs(n64 - nmx) <= 2


def test_max_weight_of_a_pass(env):
    torch, api, wl, I, w, p_lab, x1, x2 = env
    proc = api.Process.from_workload(wl)
    grid = api.Vegas(wl.ndim)
    grid.iterate(proc, N, SEED, "fp64")
    assert api.max_weight(proc) == pytest.approx(np.abs(w).max(), rel=1e-12)


@pytest.mark.parametrize("name,n", [("gg_ttx", 40_000), ("uux_ttxg", 20_000), ("gg_ttxg", 20_000),
                                    ("gg_ttxgg", 6_000)])
def test_colour_flows_of_kept_events_match_the_oracle(env, oracle_processes, tmp_path, name, n):
    torch, api = env[0], env[1]
    from oracle import unweight as uw
    from oracle import vegas as ov
    from oracle.integrand import Integrand
    from oracle.philox import vegas_uniforms
    from paper_2106_10279_gb300.process import lhe_colour_tags
    wl = W.WORKLOADS[name]
    op = oracle_processes(name)
    I = Integrand(wl, process=op)
    y = vegas_uniforms(SEED, 0, 0, 0, n, wl.ndim)
    x, jac, _ = ov.vegas_map(ov.uniform_grid(wl.ndim, wl.n_bins), y)
    w = I(x) * jac
    # a low w_max keeps many points (every point above it is kept)
    w_max = float(np.quantile(np.abs(w[w != 0]), 0.5))
    u = uw.accept_uniforms(SEED, 0, 0, n)
    keep = uw.keep(w, u, w_max)
    k = np.nonzero(keep)[0]
    if name == "gg_ttxgg":
        k = k[:300]                       # the oracle's flows are costly: the first 300 kept
    p, s_hat, x1, x2, jx, wps, ok = I.kinematics(x[:, k])
    wts = op.leading_colour_weights(p)
    pick, gap = uw.draw_flows(wts, uw.colour_uniforms(SEED, 0, 0, k))
    proc = api.Process.from_workload(wl)
    grid = api.Vegas(wl.ndim)
    tags = lhe_colour_tags(proc.desc.prog)
    lhe = api.LheWriter(tmp_path / f"{name}.lhe", [0] * len(wl.legs), [0.0] * len(wl.legs), colour_tags=tags)
    nacc, rec = api.unweight(grid, proc, n, SEED, w_max, precision="fp64", lhe=lhe)
    assert lhe.close() == nacc and nacc == int(keep.sum())
    flows = rec[:len(k), 3].astype(int)
    clear = gap > 1e-9
    assert clear.mean() > 0.99
    assert np.array_equal(flows[clear], pick[clear])
    assert np.all((flows >= 0) & (flows < tags.shape[0]))
    # every flow of the draw appears when there are many events
    if name in ("gg_ttx", "uux_ttxg"):
        assert len(set(flows.tolist())) == tags.shape[0]
    # the file's tags are the drawn flows' tags
    text = open(tmp_path / f"{name}.lhe").read()
    first = text.split("<event>\n")[1].split("</event>")[0].strip().split("\n")[1:]
    got = np.array([[int(r.split()[4]), int(r.split()[5])] for r in first])
    assert np.array_equal(got, tags[flows[0]])
