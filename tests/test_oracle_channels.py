"""The oracle's multichannel phase space (oracle/channels.py) pinned against
what the physics fixes (CPU only):

* the channel sets of the small processes, derived by hand from their
  textbook diagrams (e+e- -> mu+mu-: the s-channel photon; gg -> tt~: the
  s-channel gluon and the t- and u-channel top exchanges; uu~ -> tt~g: two
  initial-state emissions, two final-state emissions, one triple-gluon
  vertex) and the channel counts of the larger ones;
* exact momentum conservation and mass shells of every channel's points;
* each channel's density is normalised: the mean of 1/g over its unit
  hypercube is the phase-space volume, the closed form
  (2 pi)^(4-3n) (pi/2)^(n-1) s^(n-2) / ((n-1)! (n-2)!) for massless
  particles (Kleiss, Stirling & Ellis 1986) and the flat generator's volume
  for massive ones;
* the map inverts: every polar t-channel angle and every s-cluster mass read
  back from the momenta, through invariants alone, returns the unit number
  that made it;
* the partition sums to one and is, for gg -> tt~, the hand-written
  propagator products; summed over channels the estimator of the volume and
  of sigma(gg -> tt~) is unbiased (the latter against the quadrature value
  699.764 pb of test_oracle_sigma_had);
* Neyman's allocation on a hand-worked example.
"""
import math

import numpy as np
import pytest

import workloads as W
from oracle import channels as C
from oracle import phasespace as ps
from oracle.integrand import Integrand, oracle_process

R0 = 400.0   # regulators s0 = t0 (GeV^2): (pT_min)^2 of the gluon cut


def _channels(name):
    return C.derive_channels(oracle_process(W.WORKLOADS[name]))


def _final_masses(name):
    wl = W.WORKLOADS[name]
    return np.array([wl.m_top if l.particle.startswith("t") else 0.0 for l in wl.legs if not l.incoming])


def test_hand_derived_channel_sets():
    # keys: (k, masks of c_1..c_k, t-channel mass ids, #s-clusters, (mask, mass id)...)
    # final indices: e+e- -> mu+mu-: mu- 0, mu+ 1;  tt~ processes: t 0, t~ 1, g 2
    assert [c.key for c in _channels("ee_mumu")] == [(1, 3, 1, 3, -1)]
    assert [c.key for c in _channels("uux_ttx")] == [(1, 3, 1, 3, -1)]
    assert [c.key for c in _channels("gg_ttx")] == [
        (1, 3, 1, 3, -1),       # s-channel gluon
        (2, 1, 2, 0, 0),        # t-channel top: t on the side of beam a
        (2, 2, 1, 0, 0)]        # u-channel top: t~ on the side of beam a
    assert [c.key for c in _channels("uux_ttxg")] == [
        (1, 7, 2, 3, -1, 7, -1),      # g* -> g* g (triple-gluon vertex)
        (1, 7, 2, 5, 0, 7, -1),       # g* -> (t g) t~: emission from the top
        (1, 7, 2, 6, 0, 7, -1),       # g* -> t (t~ g): emission from the anti-top
        (2, 3, 4, -1, 1, 3, -1),      # emission from u~: u-quark t-channel, tt~ next to a
        (2, 4, 3, -1, 1, 3, -1)]      # emission from u: gluon next to a
    # larger processes: 18 gg -> tt~g and 159 gg -> tt~gg amplitudes, of
    # which those with a four-gluon vertex are left out and equal channels merged
    assert len(_channels("gg_ttxg")) == 15
    assert len(_channels("gg_ttxgg")) == 105


@pytest.mark.parametrize("name", ["gg_ttx", "uux_ttxg", "gg_ttxg", "gg_ttxgg"])
def test_conservation_and_mass_shells(name):
    fm = _final_masses(name)
    rng = np.random.default_rng(11)
    N = 400
    rs = np.full(N, 900.0) + 4000.0 * rng.random(N)
    for ch in _channels(name):
        assert C.n_units(ch) == 3 * len(fm) - 4
        u = rng.random((C.n_units(ch), N))
        p, inv_g, ok = C.generate(ch, u, rs, fm, R0, R0, [W.WORKLOADS[name].m_top])
        assert ok.all() and np.all(inv_g > 0) and np.all(np.isfinite(inv_g))
        tot = p.sum(axis=1)
        assert np.max(np.abs(tot[:, 0] - rs) / rs) < 1e-13
        assert np.max(np.abs(tot[:, 1:]) / rs[:, None]) < 1e-13
        m2 = p[..., 0] ** 2 - np.sum(p[..., 1:] ** 2, axis=-1)
        assert np.max(np.abs(m2 - fm ** 2) / (rs ** 2)[:, None]) < 1e-14


def _massless_volume(n, s):
    return (2 * math.pi) ** (4 - 3 * n) * (math.pi / 2) ** (n - 1) * s ** (n - 2) / (
        math.factorial(n - 1) * math.factorial(n - 2))


@pytest.mark.parametrize("name", ["gg_ttx", "uux_ttxg", "gg_ttxgg"])
def test_density_normalisation(name):
    fm = _final_masses(name)
    n = len(fm)
    rng = np.random.default_rng(5)
    N = 20000
    rs = np.full(N, 1500.0)
    chans = _channels(name)
    picks = chans if len(chans) <= 6 else [chans[i] for i in rng.choice(len(chans), 6, replace=False)]
    # flat generator's massive volume (its own normalisation is pinned in
    # test_oracle_phasespace)
    u = rng.random((3 * n - 4, 100000))
    k, wfac, _ = ps.massive(ps.massless_diet(u, np.full(100000, 1500.0)), fm, np.full(100000, 1500.0))
    w = ps.massless_weight(n, 1500.0 ** 2) * wfac
    vol_massive, err_massive = w.mean(), w.std() / math.sqrt(len(w))
    for ch in picks:
        for masses, ref, ref_err in ((np.zeros(n), _massless_volume(n, 1500.0 ** 2), 0.0),
                                     (fm, vol_massive, err_massive)):
            p, inv_g, ok = C.generate(ch, rng.random((3 * n - 4, N)), rs, masses, R0, R0, [W.WORKLOADS[name].m_top])
            est, err = inv_g.mean(), inv_g.std() / math.sqrt(N)
            assert abs(est - ref) <= 5 * math.hypot(err, ref_err) + 1e-13 * ref, (ch.key, est, err, ref)


def _mdot(a, b):
    return a[..., 0] * b[..., 0] - np.sum(a[..., 1:] * b[..., 1:], axis=-1)


def _recover(ch, p, rs, fm, masses):
    """Unit numbers read back from the momenta through invariants: the
    s-cluster masses of steps (i) and (iv) and the polar t-channel numbers
    of step (iii); returns {unit index: value}."""
    def legs(x):
        return x.legs if isinstance(x, C.Cluster) else frozenset((x,))

    def inv(X):
        Q = p[:, sorted(legs(X))].sum(axis=1)
        return _mdot(Q, Q)

    def mmin(X):
        return sum(fm[i] for i in legs(X))

    def m2(mid):
        return 0.0 if mid < 0 else masses[mid] ** 2

    def mass_u(s, lo, hi, M2):
        a = lo - M2 + R0
        return np.log((s - M2 + R0) / a) / np.log((hi - M2 + R0) / a)

    out = {}
    col = 0
    k = ch.k
    sc = [inv(c) if isinstance(c, C.Cluster) else np.full(len(rs), fm[c] ** 2) for c in ch.spine]
    if k == 1:
        sc[0] = rs ** 2
    for j, c in enumerate(ch.spine):
        if isinstance(c, C.Cluster) and k > 1:
            hi = (rs - sum(np.sqrt(sc[i]) for i in range(j)) - sum(mmin(ch.spine[i]) for i in range(j + 1, k))) ** 2
            out[col] = mass_u(sc[j], mmin(c) ** 2, hi, m2(c.mass))
            col += 1
    col += max(k - 2, 0)
    pa = np.stack([rs / 2, 0 * rs, 0 * rs, rs / 2], axis=1)
    q = pa
    for j in range(1, k):
        c = p[:, sorted(legs(ch.spine[j - 1]))].sum(axis=1)
        R = p[:, sorted(frozenset().union(*[legs(x) for x in ch.spine[j - 1:]]))].sum(axis=1)
        Rn = R - c
        # a single leg's invariant is its mass shell (not the rounding of E^2 - p^2)
        rest = frozenset().union(*[legs(x) for x in ch.spine[j:]])
        sR = _mdot(R, R)
        s_c = inv(ch.spine[j - 1]) if isinstance(ch.spine[j - 1], C.Cluster) else fm[ch.spine[j - 1]] ** 2
        sRn = _mdot(Rn, Rn) if len(rest) > 1 else fm[min(rest)] ** 2
        M = np.sqrt(sR)
        q0 = _mdot(q, R) / M
        qabs = np.sqrt(q0 ** 2 - _mdot(q, q))
        Ec = (sR + s_c - sRn) / (2 * M)
        pc = np.sqrt((sR - (np.sqrt(s_c) + np.sqrt(sRn)) ** 2) * (sR - (np.sqrt(s_c) - np.sqrt(sRn)) ** 2)) / (2 * M)
        A = m2(ch.t_mass[j - 1]) + R0 - _mdot(q, q) - s_c + 2 * q0 * Ec
        B = 2 * qabs * pc
        t = _mdot(q - c, q - c)
        out[col] = np.log((A + B) / (m2(ch.t_mass[j - 1]) + R0 - t)) / np.log((A + B) / (A - B))
        col += 2
        q = q - c

    def walk(X, sX):
        nonlocal col
        L, R = X.left, X.right
        sL = inv(L) if isinstance(L, C.Cluster) else fm[L] ** 2
        if isinstance(L, C.Cluster):
            out[col] = mass_u(sL, mmin(L) ** 2, (np.sqrt(sX) - mmin(R)) ** 2, m2(L.mass))
            col += 1
        if isinstance(R, C.Cluster):
            out[col] = mass_u(inv(R), mmin(R) ** 2, (np.sqrt(sX) - np.sqrt(sL)) ** 2, m2(R.mass))
            col += 1
        col += 2
        for Y in (L, R):
            if isinstance(Y, C.Cluster):
                walk(Y, inv(Y))

    for j, c in enumerate(ch.spine):
        if isinstance(c, C.Cluster):
            walk(c, sc[j])
    assert col == C.n_units(ch)
    return out


@pytest.mark.parametrize("name", ["gg_ttx", "uux_ttxg", "gg_ttxg", "gg_ttxgg"])
def test_map_inverts_through_invariants(name):
    fm = _final_masses(name)
    mt = W.WORKLOADS[name].m_top
    rng = np.random.default_rng(23)
    N = 300
    rs = np.full(N, 1200.0) + 3000.0 * rng.random(N)
    n_checked = 0
    for ch in _channels(name):
        u = 0.02 + 0.96 * rng.random((C.n_units(ch), N))
        p, _, ok = C.generate(ch, u, rs, fm, R0, R0, [mt])
        for col, v in _recover(ch, p, rs, fm, [mt]).items():
            assert np.max(np.abs(v - u[col])) < 1e-7, (ch.key, col)
            n_checked += 1
    assert n_checked > 0


def test_partition_of_gg_ttx_by_hand():
    chans = _channels("gg_ttx")
    mt = W.WORKLOADS["gg_ttx"].m_top
    rng = np.random.default_rng(2)
    N = 50
    rs = np.full(N, 800.0)
    fm = _final_masses("gg_ttx")
    p, _, _ = C.generate(chans[1], rng.random((2, N)), rs, fm, R0, R0, [mt])
    pa = np.stack([rs / 2, 0 * rs, 0 * rs, rs / 2], axis=1)
    a = C.partition(chans, pa, p, R0, R0, [mt])
    s = rs ** 2
    t = _mdot(pa - p[:, 0], pa - p[:, 0])
    uu = _mdot(pa - p[:, 1], pa - p[:, 1])
    P = np.stack([1 / (s + R0) ** 2, 1 / (abs(t - mt ** 2) + R0) ** 2, 1 / (abs(uu - mt ** 2) + R0) ** 2], axis=1)
    assert np.allclose(a, P / P.sum(axis=1, keepdims=True), rtol=1e-12, atol=0)
    assert np.allclose(a.sum(axis=1), 1.0, rtol=1e-14)


@pytest.mark.parametrize("name", ["uux_ttxg", "gg_ttxg"])
def test_partitioned_volume_is_unbiased(name):
    # sum_i E_i[a_i / g_i] = integral of 1 over phase space
    fm = _final_masses(name)
    mt = W.WORKLOADS[name].m_top
    chans = _channels(name)
    rng = np.random.default_rng(8)
    N = 20000
    rs = np.full(N, 1500.0)
    pa = np.stack([rs / 2, 0 * rs, 0 * rs, rs / 2], axis=1)
    tot, var = 0.0, 0.0
    for i, ch in enumerate(chans):
        p, inv_g, _ = C.generate(ch, rng.random((C.n_units(ch), N)), rs, fm, R0, R0, [mt])
        v = C.partition(chans, pa, p, R0, R0, [mt])[:, i] * inv_g
        tot += v.mean()
        var += v.var() / N
    u = rng.random((3 * len(fm) - 4, 100000))
    k, wfac, _ = ps.massive(ps.massless_diet(u, np.full(100000, 1500.0)), fm, np.full(100000, 1500.0))
    w = ps.massless_weight(len(fm), 1500.0 ** 2) * wfac
    assert abs(tot - w.mean()) < 5 * math.sqrt(var + w.var() / len(w))


def test_sigma_gg_ttx_by_channels_matches_quadrature():
    wl = W.WORKLOADS["gg_ttx"]
    I = Integrand(wl)
    chans = I.use_channels(R0, R0)
    rng = np.random.default_rng(41)
    N = 100000
    tot, var = 0.0, 0.0
    for i in range(len(chans)):
        f = I(rng.random((wl.ndim, N)), channel=i)
        tot += f.mean()
        var += f.var() / N
    err = math.sqrt(var)
    assert err < 0.01 * tot
    assert abs(tot - 699.76413) < 4 * err


def test_neyman_allocation_by_hand():
    assert C.allocate([1.0, 3.0, 0.0, 4.0], 1000, 10) == [130, 370, 10, 490]
    # shrinkage: sigma (1, 3) from 100 points each, m0 = 100: pooled variance
    # (100 + 900) / 200 = 5, shrunk deviations sqrt(3) and sqrt(7), so the
    # shares are sqrt(3) / (sqrt(3) + sqrt(7)) = 0.39564.. and 0.60435..
    assert C.allocate([1.0, 3.0], 1000, 0, n_prev=[100, 100], m0=100.0) == [395, 604]
    # with m0 = 0 the shrinkage is the identity; with no points, the pooled deviation
    assert C.allocate([1.0, 3.0], 1000, 0, n_prev=[50, 70], m0=0.0) == [250, 750]
    assert C.allocate([1.0, 3.0], 1000, 0, n_prev=[0, 100], m0=10.0) == [500, 500]
    assert C.allocate([0.0, 0.0, 0.0], 100, 5) == [33, 33, 33]
    assert C.allocate([2.0], 4096, 4096) == [4096]
    with pytest.raises(ValueError):
        C.allocate([1.0, 1.0], 10, 8)


def test_channel_gradient_matches_central_differences():
    # the oracle's dual-number derivative of a channel's integrand with
    # respect to the unit numbers and the top mass, against central
    # differences (gg -> tt~ has no cuts: the integrand is smooth)
    wl = W.WORKLOADS["gg_ttx"]
    I = Integrand(wl)
    I.use_channels(R0, R0)
    x = 0.1 + 0.8 * W.uniform_points(wl.ndim, 5, 3)
    h = 1e-6
    for ch in range(3):
        f, dfdx, dfdm = I.gradient(x, channel=ch)
        assert np.allclose(f, I(x, channel=ch), rtol=1e-13, atol=0)
        for j in range(wl.ndim):
            xp, xm = x.copy(), x.copy()
            xp[j] += h
            xm[j] -= h
            fd = (I(xp, channel=ch) - I(xm, channel=ch)) / (2 * h)
            assert np.allclose(dfdx[j], fd, rtol=2e-6, atol=1e-9 * np.abs(f).max()), (ch, j)
        Ip = Integrand(wl, m_top=wl.m_top + 1e-4)
        Im = Integrand(wl, m_top=wl.m_top - 1e-4)
        Ip.use_channels(R0, R0)
        Im.use_channels(R0, R0)
        fd = (Ip(x, channel=ch) - Im(x, channel=ch)) / 2e-4
        assert np.allclose(dfdm, fd, rtol=1e-5, atol=1e-9 * np.abs(f).max()), ch
