"""Pins of the oracle's observable histograms (oracle/observables.py):

* the observables of hand-built momenta: pT, rapidity and pseudorapidity of
  a particle of known transverse mass and rapidity, and of a massless one
  (where eta = y);
* the collider-frame boost adds the pair rapidity to every rapidity;
* bins and per-bin sums on a small hand-worked example, and the sums over a
  range holding every point equal the pass's integral estimate;
* physics: in e+e- -> mu+mu- through a photon, dsigma/dcos(theta) is
  (3 sigma / 8)(1 + cos^2 theta), so the mu- pseudorapidity histogram is
  (3 sigma / 8) [tanh eta + tanh^3 eta / 3] between the bin edges, with
  sigma = 4 pi alpha^2 / (3 s); the oracle's histogram of 2e5 uniform points
  agrees bin by bin within 5 of its own Monte Carlo errors.
"""
import math

import numpy as np
import pytest

import workloads as W
from oracle import observables as ob
from oracle import unweight as uw


def test_values_of_hand_built_momenta():
    pt, y, m = 40.0, 0.7, 173.0
    mt = math.hypot(m, pt)
    phi = 0.3
    p = np.array([[[0.0] * 4, [mt * math.cosh(y), pt * math.cos(phi), pt * math.sin(phi), mt * math.sinh(y)]]])
    assert ob.values(p, ob.PT, 1)[0] == pytest.approx(pt, rel=1e-14)
    assert ob.values(p, ob.RAPIDITY, 1)[0] == pytest.approx(y, rel=1e-13)
    # pseudorapidity of a massive particle: asinh(pz / pT) with pz = mT sinh y
    assert ob.values(p, ob.PSEUDORAPIDITY, 1)[0] == pytest.approx(math.asinh(mt * math.sinh(y) / pt), rel=1e-14)
    # massless: eta = y
    q = np.array([[[pt * math.cosh(y), pt, 0.0, pt * math.sinh(y)]]])
    assert ob.values(q, ob.PSEUDORAPIDITY, 0)[0] == pytest.approx(y, rel=1e-13)
    assert ob.values(q, ob.RAPIDITY, 0)[0] == pytest.approx(y, rel=1e-13)
    # transverse, at rest along z: y = eta = 0
    r = np.array([[[5.0, 3.0, 4.0, 0.0]]])
    assert ob.values(r, ob.PT, 0)[0] == 5.0
    assert ob.values(r, ob.RAPIDITY, 0)[0] == 0.0
    assert ob.values(r, ob.PSEUDORAPIDITY, 0)[0] == 0.0


def test_collider_boost_shifts_rapidities():
    rng = np.random.default_rng(4)
    n = 50
    m = 173.0
    pt = rng.uniform(1, 300, n)
    y = rng.uniform(-2, 2, n)
    phi = rng.uniform(0, 2 * np.pi, n)
    mt = np.hypot(m, pt)
    p = np.zeros((n, 1, 4))
    p[:, 0] = np.stack([mt * np.cosh(y), pt * np.cos(phi), pt * np.sin(phi), mt * np.sinh(y)], axis=1)
    x1 = rng.uniform(0.01, 0.5, n)
    x2 = rng.uniform(0.01, 0.5, n)
    lab = uw.lab_frame(p, x1, x2)
    yb = 0.5 * (np.log(x1) - np.log(x2))
    assert np.allclose(ob.values(lab, ob.RAPIDITY, 0), y + yb, rtol=0, atol=1e-12)
    assert np.allclose(ob.values(lab, ob.PT, 0), pt, rtol=1e-13, atol=0)


def test_bins_and_sums_by_hand():
    v = np.array([0.05, 0.25, 0.95, 1.0, -0.1, 0.30])
    b = ob.bin_index(v, 4, 0.0, 1.0)
    assert b.tolist() == [0, 1, 3, -1, -1, 1]
    w = np.array([1.0, 2.0, 3.0, 4.0, 5.0, -1.0])
    sigma, err, count = ob.histogram(w, b, 4, 6)
    assert count.tolist() == [1, 2, 0, 1]
    assert np.allclose(sigma, [1 / 6, 1 / 6, 0.0, 3 / 6], rtol=1e-15, atol=0)
    # bin 1: sum w = 1, sum w^2 = 5 -> var = (5/6 - 1/36) / 5
    assert err[1] == pytest.approx(math.sqrt((5 / 6 - 1 / 36) / 5), rel=1e-14)
    assert err[2] == 0.0


def test_full_range_adds_up_to_the_integral(oracle_processes):
    from oracle.integrand import Integrand
    wl = W.GG_TTX
    I = Integrand(wl, process=oracle_processes("gg_ttx"))
    x = W.uniform_points(wl.ndim, 3000, 17)
    p, s_hat, x1, x2, jx, wps, ok = I.kinematics(x)
    passing = ok & I.cuts(p)
    w = I(x)
    lab = uw.lab_frame(p, x1, x2)
    (sig_pt, _, c_pt), (sig_y, _, c_y) = ob.histograms(lab, passing, w, [(ob.PT, 2, 20, 0.0, 13000.0),
                                                                        (ob.RAPIDITY, 2, 25, -20.0, 20.0)])
    assert c_pt.sum() == passing.sum() == c_y.sum()
    assert np.sum(sig_pt) == pytest.approx(w.mean(), rel=1e-13)
    assert np.sum(sig_y) == pytest.approx(w.mean(), rel=1e-13)


def test_ee_mumu_pseudorapidity_is_the_photon_distribution(oracle_processes):
    from oracle.integrand import Integrand
    wl = W.EE_MUMU
    I = Integrand(wl, process=oracle_processes("ee_mumu"))
    n = 200_000
    x = W.uniform_points(wl.ndim, n, 5)
    p, s_hat, x1, x2, jx, wps, ok = I.kinematics(x)
    w = I(x)
    lab = uw.lab_frame(p, x1, x2)
    # the outgoing mu-: the first final-state leg of the workload
    leg = 2
    assert wl.legs[leg].particle in ("mu-", "m-", "mu")
    nb, lo, hi = 12, -3.0, 3.0
    ((sigma, err, count),) = ob.histograms(lab, ok, w, [(ob.PSEUDORAPIDITY, leg, nb, lo, hi)])
    s = (W.SQRT_S_EE) ** 2
    sig_tot = 4 * math.pi * W.ALPHA_EM ** 2 / (3 * s) * W.GEV2_TO_PB
    edges = np.linspace(lo, hi, nb + 1)
    F = lambda e: 3 * sig_tot / 8 * (np.tanh(e) + np.tanh(e) ** 3 / 3)
    ref = F(edges[1:]) - F(edges[:-1])
    assert np.all(count > 0)
    assert np.all(np.abs(sigma - ref) <= 5 * err), (sigma, ref, err)
