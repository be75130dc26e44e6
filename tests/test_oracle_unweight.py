"""Pins of the oracle's unweighting and event frame (CPU only)."""
import numpy as np
import pytest

import workloads as W
from oracle import unweight as uw
from oracle.philox import vegas_uniforms

MDOT = np.array([1.0, -1.0, -1.0, -1.0])


def test_accept_uniforms_are_a_separate_philox_stream():
    # block 15 of the same counters the points use: not one of the point's
    # own numbers, uniform in (0, 1)
    u = uw.accept_uniforms(7, 2, 1, 20000)
    y = vegas_uniforms(7, 2, 1, 0, 20000, 20)
    assert not np.any(np.isin(u, y))
    assert np.all((u > 0) & (u < 1))
    assert abs(u.mean() - 0.5) < 5 * np.sqrt(1 / 12 / 20000)


def test_unweighting_is_unbiased_and_flat():
    # expected sum of event weights = mean weight; below w_max the kept
    # fraction of a bin is w / w_max
    rng = np.random.default_rng(3)
    N = 400_000
    w = rng.exponential(1.0, N)
    w_max = 3.0
    u = rng.random(N)
    k = uw.keep(w, u, w_max)
    ew = uw.event_weights(w[k], w_max, N)
    est = ew.sum()
    # variance of the unweighted estimator per point: E[max(w,wmax)^2 1_keep]/N^2 ...
    var = (np.mean(np.where(k, np.maximum(w, w_max) ** 2, 0.0)) - est ** 2) / N
    assert abs(est - w.mean()) < 5 * np.sqrt(var)
    below = (w > 0.9) & (w < 1.1)
    assert abs(k[below].mean() - 1.0 / w_max) < 0.01
    assert np.all(k[w > w_max])                     # overweight points are always kept
    assert np.allclose(ew[w[k] > w_max] * N, w[k][w[k] > w_max])


def test_lab_frame_boost():
    # incoming partons end up with x1 E_beam along +z and x2 E_beam along -z;
    # invariant masses and transverse momenta unchanged
    rng = np.random.default_rng(4)
    N = 100
    x1, x2 = rng.uniform(0.01, 0.9, N), rng.uniform(0.01, 0.9, N)
    S = 13000.0 ** 2
    rs = np.sqrt(x1 * x2 * S)
    p = np.zeros((N, 3, 4))
    p[:, 0] = np.stack([rs / 2, 0 * rs, 0 * rs, rs / 2], 1)
    p[:, 1] = np.stack([rs / 2, 0 * rs, 0 * rs, -rs / 2], 1)
    p[:, 2] = np.stack([rs, rng.normal(size=N), rng.normal(size=N), rng.normal(size=N)], 1)
    q = uw.lab_frame(p, x1, x2)
    assert np.allclose(q[:, 0, 0], x1 * 6500.0, rtol=1e-13)
    assert np.allclose(q[:, 0, 3], x1 * 6500.0, rtol=1e-13)
    assert np.allclose(q[:, 1, 0], x2 * 6500.0, rtol=1e-13)
    assert np.allclose(q[:, 1, 3], -x2 * 6500.0, rtol=1e-13)
    m2 = lambda a: np.einsum("nm,m,nm->n", a, MDOT, a)
    assert np.allclose(m2(q[:, 2]), m2(p[:, 2]), rtol=1e-10, atol=1e-8)
    assert np.array_equal(q[:, :, 1:3], p[:, :, 1:3])


# ------------------------------------------------------------ colour flows
def test_colour_tags_of_gg_to_ttbar():
    # (t^a1 t^a2)_{t, tbar}: the top's colour line runs through gluon 1 then
    # gluon 2 into the antitop; incoming gluons carry colour and anticolour
    # swapped with respect to the all-outgoing assignment
    from oracle.integrand import oracle_process
    from oracle.unweight import colour_tags
    op = oracle_process(W.GG_TTX)
    tags = colour_tags(op.string_labels(), op.legs)
    assert tags.tolist() == [[[501, 502], [502, 503], [501, 0], [0, 503]],
                             [[502, 503], [501, 502], [501, 0], [0, 503]]]
    op = oracle_process(W.UUX_TTX)
    tags = colour_tags(op.string_labels(), op.legs)
    # u u~ -> t t~: annihilation lines (u with u~, t with t~) and exchange
    # lines (u's colour into t, u~'s anticolour into t~)
    assert tags.tolist() == [[[501, 0], [0, 501], [502, 0], [0, 502]],
                             [[502, 0], [0, 501], [502, 0], [0, 501]]]


@pytest.mark.parametrize("name", ["ee_mumu", "gg_ttx", "uux_ttx", "gg_ttxg", "uux_ttxg", "gg_ttxgg"])
def test_colour_tags_conserve_colour(name):
    # every line appears once as an outgoing colour or incoming anticolour and
    # once as an outgoing anticolour or incoming colour; gluons carry both,
    # (anti)quarks one, colourless particles none
    from oracle.integrand import oracle_process
    from oracle.unweight import colour_tags
    from oracle.feynman import PARTICLES, COLOUR_DIM
    wl = W.WORKLOADS[name]
    op = oracle_process(wl)
    tags = colour_tags(op.string_labels(), op.legs)
    assert tags.shape[0] == op.string_basis().shape[1]
    for t in tags:
        src, snk = [], []
        for i, (part, inc) in enumerate(op.legs):
            c, a = t[i]
            dim = COLOUR_DIM[PARTICLES[part][1]]
            assert int(c != 0) + int(a != 0) == {1: 0, 3: 1, 8: 2}[dim]
            (snk if inc else src).append(c)
            (src if inc else snk).append(a)
        src = sorted(v for v in src if v)
        snk = sorted(v for v in snk if v)
        assert src == snk and len(set(src)) == len(src)


def test_flow_draw_follows_the_weights():
    from oracle.unweight import colour_uniforms, draw_flows
    wts = np.array([[0.0, 1.0, 3.0, 0.0, 6.0]] * 200_000)
    pick, gap = draw_flows(wts, colour_uniforms(5, 2, 1, np.arange(200_000)))
    freq = np.bincount(pick, minlength=5) / 200_000
    assert freq[0] == 0 and freq[3] == 0
    assert np.allclose(freq, [0, 0.1, 0.3, 0, 0.6], atol=0.005)


@pytest.mark.parametrize("name", ["gg_ttx", "uux_ttxg"])
def test_leading_colour_weights_sum_to_the_leading_colour_msq(name):
    from oracle.integrand import Integrand
    wl = W.WORKLOADS[name]
    I = Integrand(wl)
    x = W.uniform_points(wl.ndim, 20, 3)
    p, s_hat, x1, x2, jx, wps, ok = I.kinematics(x)
    w = I.proc.leading_colour_weights(p)
    assert np.allclose(w.sum(axis=1), I.proc.msq_leading_colour(p), rtol=1e-13, atol=0)
    assert np.all(w >= 0)
