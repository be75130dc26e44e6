"""Pins of the oracle's phase space and x1, x2 map (CPU only)."""
import math

import numpy as np
import pytest
from scipy import integrate, stats

from oracle import phasespace as ps

MDOT = np.array([1.0, -1.0, -1.0, -1.0])


def test_massless_volume_closed_forms():
    # (2pi)^(4-3n) (pi/2)^(n-1) s^(n-2) / ((n-1)!(n-2)!): 1/(8 pi), s/(256 pi^3), ...
    assert ps.massless_weight(2, 1.0) == pytest.approx(1 / (8 * math.pi), rel=1e-15)
    assert ps.massless_weight(3, 1.0) == pytest.approx(1 / (256 * math.pi ** 3), rel=1e-15)
    assert ps.massless_weight(2, 1.0) == pytest.approx(0.0397887, rel=1e-6)
    assert ps.massless_weight(3, 1.0) == pytest.approx(1.259826e-4, rel=1e-6)
    assert ps.massless_weight(4, 1.0) == pytest.approx(1.329656e-7, rel=1e-6)


@pytest.mark.parametrize("n", [2, 3, 4])
def test_diet_momentum_conservation_and_massless(n):
    rng = np.random.default_rng(n)
    u = rng.random((3 * n - 4, 2000))
    rs = rng.uniform(100, 5000, 2000)
    p = ps.massless_diet(u, rs)
    tot = p.sum(axis=1)
    assert np.max(np.abs(tot[:, 0] - rs) / rs) < 1e-13
    assert np.max(np.abs(tot[:, 1:]) / rs[:, None]) < 1e-13
    m2 = np.einsum("nkm,m,nkm->nk", p, MDOT, p)
    assert np.max(np.abs(m2) / rs[:, None] ** 2) < 1e-13
    assert np.all(p[:, :, 0] > 0)


@pytest.mark.parametrize("n", [3, 4])
def test_diet_is_flat_energy_spectrum(n):
    # flat massless n-body phase space: z = 2E/sqrt(s) of any one particle has
    # density (n-1)(n-2) z (1-z)^(n-3) on [0, 1]
    rng = np.random.default_rng(10 + n)
    N = 40000
    p = ps.massless_diet(rng.random((3 * n - 4, N)), 1.0)
    for i in range(n):
        z = 2 * p[:, i, 0]
        if n == 3:
            cdf = lambda t: t * t
        else:
            cdf = lambda t: 3 * t * t - 2 * t ** 3
        assert stats.kstest(z, cdf).pvalue > 1e-3
        assert abs(np.mean(p[:, i, 0]) - 1.0 / n) < 5 * np.std(p[:, i, 0]) / math.sqrt(N)


def test_diet_matches_classic_rambo_distribution():
    n = 4
    rng = np.random.default_rng(21)
    N = 30000
    a = ps.massless_diet(rng.random((3 * n - 4, N)), 1.0)
    b = ps.rambo_classic(rng.random((4 * n, N)), 1.0, n)
    for i in range(n):
        for obs in (lambda q: q[:, i, 0], lambda q: q[:, i, 3],
                    lambda q: np.hypot(q[:, i, 1], q[:, i, 2])):
            assert stats.ks_2samp(obs(a), obs(b)).pvalue > 1e-3
    # pair invariant
    s01a = 2 * np.einsum("nm,m,nm->n", a[:, 0], MDOT, a[:, 1])
    s01b = 2 * np.einsum("nm,m,nm->n", b[:, 0], MDOT, b[:, 1])
    assert stats.ks_2samp(s01a, s01b).pvalue > 1e-3
    assert abs(np.mean(s01a) - 1 / 6) < 0.01


def test_massive_two_body_weight_is_beta_over_8pi():
    rng = np.random.default_rng(3)
    rs = rng.uniform(350, 3000, 500)
    p = ps.massless_diet(rng.random((2, 500)), rs)
    k, wfac, ok = ps.massive(p, [173.0, 173.0], rs)
    beta = np.sqrt(1 - 4 * 173.0 ** 2 / rs ** 2)
    w = ps.massless_weight(2, rs ** 2) * wfac
    assert np.max(np.abs(w / (beta / (8 * math.pi)) - 1)) < 1e-13
    # unequal masses: beta = lambda^(1/2)(s, m1^2, m2^2)/s
    k, wfac, ok = ps.massive(p, [173.0, 50.0], rs)
    s = rs ** 2
    lam = (s - (173 + 50) ** 2) * (s - (173 - 50) ** 2)
    w = ps.massless_weight(2, s) * wfac
    assert np.max(np.abs(w / (np.sqrt(lam) / s / (8 * math.pi)) - 1)) < 1e-13


def test_massive_on_shell_and_conserved():
    rng = np.random.default_rng(4)
    rs = rng.uniform(400, 3000, 1000)
    m = np.array([173.0, 173.0, 0.0, 0.0])
    p = ps.massless_diet(rng.random((8, 1000)), rs)
    k, wfac, ok = ps.massive(p, m, rs)
    tot = k.sum(axis=1)
    assert np.max(np.abs(tot[:, 0] - rs) / rs) < 1e-14
    assert np.max(np.abs(tot[:, 1:]) / rs[:, None]) < 1e-13
    m2 = np.einsum("nkm,m,nkm->nk", k, MDOT, k)
    assert np.max(np.abs(m2 - m ** 2) / rs[:, None] ** 2) < 1e-12


def test_massive_three_body_volume_matches_dalitz_integral():
    # Phi_3 = 1/(128 pi^3 s) * Dalitz area; the RAMBO weight average over flat
    # massless points estimates it
    rs = 800.0
    s = rs * rs
    m1, m2, m3 = 173.0, 173.0, 0.0

    def s23_range(s12):
        e2 = (s12 - m1 ** 2 + m2 ** 2) / (2 * math.sqrt(s12))
        e3 = (s - s12 - m3 ** 2) / (2 * math.sqrt(s12))
        p2 = math.sqrt(max(e2 * e2 - m2 * m2, 0))
        p3 = math.sqrt(max(e3 * e3 - m3 * m3, 0))
        return (e2 + e3) ** 2 - (p2 + p3) ** 2, (e2 + e3) ** 2 - (p2 - p3) ** 2

    area, _ = integrate.quad(lambda s12: s23_range(s12)[1] - s23_range(s12)[0],
                             (m1 + m2) ** 2, (rs - m3) ** 2, limit=200)
    vol = area / (128 * math.pi ** 3 * s)
    rng = np.random.default_rng(8)
    N = 400000
    p = ps.massless_diet(rng.random((5, N)), rs)
    k, wfac, ok = ps.massive(p, [m1, m2, m3], rs)
    w = ps.massless_weight(3, s) * wfac
    est, err = np.mean(w), np.std(w) / math.sqrt(N)
    assert abs(est - vol) < 4 * err
    assert err / vol < 3e-3


def test_xmap_jacobian_integrates_luminosity_measure():
    # int dx1 dx2 theta(x1 x2 > tau_min) h(x1, x2) = int dy1 dy2 J h(x1(y), x2(y))
    tau_min = 7.0838e-4
    h = lambda x1, x2: x1 ** 0.3 * (1 - x2) ** 2
    ref, _ = integrate.dblquad(lambda x2, x1: h(x1, x2), tau_min, 1,
                               lambda x1: tau_min / x1, lambda x1: 1, epsabs=1e-13, epsrel=1e-11)
    g, w = np.polynomial.legendre.leggauss(80)
    y = 0.5 * (g + 1)
    wy = 0.5 * w
    Y1, Y2 = np.meshgrid(y, y, indexing="ij")
    x1, x2, tau, jac = ps.xmap(Y1.ravel(), Y2.ravel(), tau_min)
    val = np.sum((wy[:, None] * wy[None, :]).ravel() * jac * h(x1, x2))
    assert abs(val / ref - 1) < 1e-9
    assert np.allclose(x1 * x2, tau, rtol=1e-15)
    assert np.all((x1 >= tau_min) & (x1 <= 1) & (x2 >= tau_min) & (x2 <= 1))


@pytest.mark.parametrize("m", [2, 3, 4])
def test_mass_ratio_root_full_precision_near_both_ends(m):
    # the root of F(x) = m x^(m-1) - (m-1) x^m = r, returned as a double x:
    # the residual of the form solved must vanish to rounding plus the change
    # of that residual over one ulp of x, including r -> 1 (x -> 1, measured
    # in d = 1 - x, exact for x >= 1/2, through 1 - F(1 - d) = 1 - r)
    r = np.array([1e-14, 1e-9, 0.25, 0.5, 0.75, 1 - 1e-9, 1 - 1e-13])
    x = ps._mass_ratio(r, m)
    u = np.spacing(x)
    F = lambda t: m * t ** (m - 1) - (m - 1) * t ** m
    coef = [(m - 1) * math.comb(m, k) - m * math.comb(m - 1, k) for k in range(m + 1)]
    G = lambda d: sum(coef[k] * (-d) ** k for k in range(2, m + 1))
    low = r <= 0.5
    eps = np.finfo(float).eps
    res_lo = np.abs(F(x) - r)
    tol_lo = 4 * eps * r + np.abs(F(x + u) - F(x))
    assert np.all(res_lo[low] <= tol_lo[low])
    d = 1.0 - x
    res_hi = np.abs(G(d) - (1 - r))
    tol_hi = 4 * eps * (1 - r) + np.abs(G(d + u) - G(d))
    assert np.all(res_hi[~low] <= tol_hi[~low])
    # and 1 - x is resolved far beyond sqrt(eps): against the m = 2 closed form
    if m == 2:
        assert np.all(np.abs(d[~low] - np.sqrt(1 - r[~low])) <= 2 * u[~low])


def test_daughter_energy_keeps_precision_at_mass_ratio_near_one():
    # first decay of n = 3 in the CM frame: the massless daughter has
    # E = sqrt(s)(1 - x)/2 with 1 - x = sqrt(1 - r) (m = 2 closed form); for r
    # next to 1 it is ~1e-6 sqrt(s) and must still be exact to rounding
    r = np.array([0.5, 0.9, 1 - 1e-9, 1 - 1e-12, 1 - 2.0 ** -52])
    N = r.size
    u = np.vstack([np.full(N, 0.3), np.full(N, 0.6), r, np.full(N, 0.7), np.full(N, 0.2)])
    rs = 1000.0
    p = ps.massless_diet(u, rs)
    e = p[:, 0, 0]
    assert np.all(np.abs(e / (rs * np.sqrt(1 - r) / 2) - 1) <= 4 * np.finfo(float).eps)
    assert np.max(np.abs(p.sum(axis=1)[:, 0] - rs)) <= 4e-13 * rs
