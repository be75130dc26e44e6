"""Pins of the oracle's integrand assembly and Vegas (CPU only)."""
import math

import numpy as np
import pytest

import workloads as W
from oracle import vegas
from oracle.integrand import Integrand

SIGMA_EE_PB = 4 * math.pi * W.ALPHA_EM ** 2 / (3 * W.SQRT_S_EE ** 2) * W.GEV2_TO_PB


def test_ee_cross_section_constant():
    assert SIGMA_EE_PB == pytest.approx(12.0215046, rel=1e-8)


def test_ee_integrand_angular_integral_is_total_cross_section():
    I = Integrand(W.EE_MUMU)
    g, w = np.polynomial.legendre.leggauss(40)
    y = 0.5 * (g + 1)
    Y1, Y2 = np.meshgrid(y, y, indexing="ij")
    wts = np.outer(0.5 * w, 0.5 * w).ravel()
    f = I(np.stack([Y1.ravel(), Y2.ravel()]))
    assert np.sum(wts * f) == pytest.approx(SIGMA_EE_PB, rel=1e-13)


def test_hadronic_integrand_assembly_against_partonic_closed_form():
    # at fixed (y1, y2) the angular integral of f equals
    # J_x f_g(x1) f_g(x2) sigma-hat(gg -> tt~)(s-hat) in pb
    wl = W.GG_TTX
    I = Integrand(wl)
    # f does not depend on phi for 2 -> 2; the cos-theta integrand has poles
    # at +-1/beta, close to the interval at large s-hat: many nodes
    g, w = np.polynomial.legendre.leggauss(400)
    C = 0.5 * (g + 1)
    P = np.full_like(C, 0.37)
    wts = 0.5 * w
    m, a_s = wl.m_top, wl.alpha_s
    for y1, y2 in ((0.9, 0.5), (0.6, 0.2), (0.3, 0.77)):
        n = C.size
        x = np.stack([np.full(n, y1), np.full(n, y2), C.ravel(), P.ravel()])
        f, parts = I(x, return_parts=True)
        val = np.sum(wts * f)
        s = parts["s_hat"][0]
        x1, x2, jx = parts["x1"][0], parts["x2"][0], parts["jx"][0]
        rho = 4 * m * m / s
        b = math.sqrt(1 - rho)
        sig = math.pi * a_s ** 2 / (3 * s) * ((1 + rho + rho ** 2 / 16) * math.log((1 + b) / (1 - b))
                                              - b * (7 / 4 + 31 * rho / 16))
        lum = I.pdfs[0].f(x1, wl.mu_f2)[0] * I.pdfs[1].f(x2, wl.mu_f2)[0]
        assert val == pytest.approx(jx * lum * sig * W.GEV2_TO_PB, rel=1e-12)


def test_cuts_on_constructed_momenta():
    I = Integrand(W.GG_TTXGG)
    p = np.zeros((4, 6, 4))
    def gluon(pt, y, phi):
        return np.array([pt * math.cosh(y), pt * math.cos(phi), pt * math.sin(phi), pt * math.sinh(y)])
    # event 0: both gluons hard and separated -> kept
    p[0, 4], p[0, 5] = gluon(50, 0.0, 0.0), gluon(60, 0.2, 1.0)
    # event 1: one gluon below 20 GeV -> cut
    p[1, 4], p[1, 5] = gluon(19.9, 0.0, 0.0), gluon(60, 0.2, 1.0)
    # event 2: Delta R = 0.3 -> cut
    p[2, 4], p[2, 5] = gluon(50, 0.0, 0.0), gluon(60, 0.3, 0.0)
    # event 3: Delta phi wraps across pi: phi = 3.1 and -3.1 -> Delta R ~ 0.083 -> cut
    p[3, 4], p[3, 5] = gluon(50, 1.0, 3.1), gluon(60, 1.0, -3.1)
    assert I.cuts(p).tolist() == [True, False, False, False]


# --------------------------------------------------------------- Vegas
def test_vegas_map_is_measure_preserving():
    rng = np.random.default_rng(1)
    grid = np.sort(np.concatenate([[[0.0]] * 3, rng.random((3, 9)), [[1.0]] * 3], axis=1), axis=1)
    g, w = np.polynomial.legendre.leggauss(30)
    # in one dimension: int_0^1 J(y) h(x(y)) dy = int_0^1 h(x) dx, bin by bin
    h = lambda x: np.cos(3 * x) + x ** 2
    tot = 0.0
    for i in range(10):
        y = (i + 0.5 * (g + 1)) / 10
        x, jac, bins = vegas.vegas_map(grid[:1], y[None, :])
        tot += np.sum(0.05 * w * jac * h(x[0]))
    ref = math.sin(3) / 3 + 1 / 3
    assert tot == pytest.approx(ref, rel=1e-13)


def test_vegas_uniform_d_is_a_fixed_point_of_refinement():
    grid = vegas.uniform_grid(2, 20)
    new = vegas.refine(grid, np.full((2, 20), 3.0), n=10)
    assert np.allclose(new, grid, atol=1e-15)


def test_vegas_constant_integrand_grid_moves_only_by_fluctuations():
    # d_i = sum of w^2 = bin count for f = 1: the grid only follows the
    # Poisson fluctuations of the counts, damped by the compression
    res = vegas.run(lambda x: np.ones(x.shape[1]), ndim=3, n_events=200000, n_iter=3, seed=5, nbins=20)
    assert np.max(np.abs(res["grid"] - vegas.uniform_grid(3, 20))) < 5e-3
    assert res["sigma"] == pytest.approx(1.0, abs=1e-12)


def test_vegas_combination_closed_form():
    mean, err, chi2 = vegas.combine([(1.0, 0.1), (1.2, 0.2)])
    w1, w2 = 100.0, 25.0
    assert mean == pytest.approx((w1 * 1.0 + w2 * 1.2) / (w1 + w2), rel=1e-15)
    assert err == pytest.approx(1 / math.sqrt(w1 + w2), rel=1e-15)
    assert chi2 == pytest.approx(w1 * (1.0 - mean) ** 2 + w2 * (1.2 - mean) ** 2, rel=1e-12)


def test_vegas_refine_hand_example():
    # 4 bins, all of d in bin 0: smoothed (1/2, 1/3, 0, 0) -> r = (0.6, 0.4, 0, 0)
    grid = vegas.uniform_grid(1, 4)
    d = np.array([[8.0, 0.0, 0.0, 0.0]])
    new = vegas.refine(grid, d, n=2, alpha=1.0)
    r = np.array([0.6, 0.4])
    comp = (r - 1) / np.log(r)
    per = comp.sum() / 4
    e1 = per / comp[0] * 0.25
    e2 = 2 * per / comp[0] * 0.25
    e3 = 0.25 + (3 * per - comp[0]) / comp[1] * 0.25
    assert np.allclose(new[0], [0, e1, e2, e3, 1], rtol=1e-14)


def test_vegas_separable_integrand_converges_and_adapts():
    # f = prod_j 3 exp(-3 x_j)/(1 - e^-3): integral 1, peaked at x = 0
    c = 3.0 / (1 - math.exp(-3.0))
    f = lambda x: np.prod(c * np.exp(-3.0 * x), axis=0)
    res = vegas.run(f, ndim=3, n_events=20000, n_iter=6, seed=2, nbins=30)
    assert abs(res["sigma"] - 1.0) < 4 * res["error"]
    first_err = res["iterations"][0][1]
    last_err = res["iterations"][-1][1]
    assert last_err < 0.5 * first_err
    assert res["grid"][0, 15] < 0.35            # bins crowd towards x = 0


def test_vegas_ee_cross_section():
    I = Integrand(W.EE_MUMU)
    res = vegas.run(I, ndim=2, n_events=20000, n_iter=4, seed=1, nbins=50)
    assert abs(res["sigma"] - SIGMA_EE_PB) < 4 * res["error"]
    assert res["error"] / res["sigma"] < 2e-3


def test_vegas_histogram_counts_sum_to_events():
    res = vegas.run(lambda x: x[0] + x[1], ndim=2, n_events=5000, n_iter=2, seed=9, nbins=10)
    for dsum, cnt, grid in res["hist"]:
        assert np.all(cnt.sum(axis=1) == 5000)


def test_helicity_sampling_is_unbiased(oracle_processes):
    # averaging the sampled integrand over the helicity choice gives the full
    # helicity sum exactly; over random seeds, within the sampling spread
    import workloads as W
    from oracle.integrand import Integrand
    wl = W.GG_TTX
    I = Integrand(wl, process=oracle_processes("gg_ttx"))
    hels = I.nonzero_helicities()
    # gg -> tt~: the four assignments with equal gluon helicities and opposite
    # top helicities vanish
    assert len(hels) == 12
    assert all(not (h[0] == h[1] and h[2] != h[3]) for h in hels)
    # massless e+e- -> mu+mu- through a photon: 4 of 16 survive (chirality)
    assert len(Integrand(W.EE_MUMU, process=oracle_processes("ee_mumu")).nonzero_helicities()) == 4
    x = W.uniform_points(wl.ndim, 40, 5)
    full = I(x)
    # every helicity choice in turn: their mean is the full sum
    nh = len(hels)
    mean = sum(I.sampled(x, 0, hels, pick=np.full(40, h))[0] for h in range(nh)) / nh
    nz = full != 0
    assert np.all((mean == 0) == (full == 0))
    assert np.max(np.abs(mean[nz] / full[nz] - 1)) < 1e-13
    # the Philox choice is uniform over the list
    _, pick = I.sampled(W.uniform_points(wl.ndim, 4000, 6), 3, hels)
    counts = np.bincount(pick, minlength=nh)
    assert counts.sum() == 4000 and np.all(np.abs(counts - 4000 / nh) < 5 * np.sqrt(4000 / nh))


def test_helicity_pair_sampling_is_unbiased(oracle_processes):
    # pairs of the kept helicities that differ at one leg: averaging the
    # pair-sampled integrand over the pair choice gives the full helicity sum
    # exactly; gg -> tt~ paired at the antitop: the 12 kept rows form 8 pairs,
    # 4 of them with one member (equal gluon helicities keep only equal top
    # helicities)
    import workloads as W
    from oracle.integrand import Integrand
    wl = W.GG_TTX
    I = Integrand(wl, process=oracle_processes("gg_ttx"))
    hels = I.nonzero_helicities()
    pairs = Integrand.helicity_pairs(hels, 3)
    assert len(pairs) == 8
    assert sum(1 for a, b in pairs if a is None or b is None) == 4
    assert sorted(h for q in pairs for h in q if h is not None) == sorted(tuple(h) for h in hels)
    for a, b in pairs:
        if a is not None and b is not None:
            assert a[:3] == b[:3] and (a[3], b[3]) == (-1, 1)
    x = W.uniform_points(wl.ndim, 40, 5)
    full = I(x)
    mean = sum(I.sampled_pairs(x, 0, pairs, pick=np.full(40, u))[0] for u in range(8)) / 8
    nz = full != 0
    assert np.all((mean == 0) == (full == 0))
    assert np.max(np.abs(mean[nz] / full[nz] - 1)) < 1e-13
    # the same Philox draw as single-helicity sampling, over the pair list
    _, pick = I.sampled_pairs(W.uniform_points(wl.ndim, 4000, 6), 3, pairs)
    counts = np.bincount(pick, minlength=8)
    assert counts.sum() == 4000 and np.all(np.abs(counts - 500) < 5 * np.sqrt(500))
