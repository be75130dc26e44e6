"""The oracle's forward-mode dual numbers and its integrand gradient (CPU).

* the dual-number rules against derivatives known in closed form;
* implicit derivatives of the roots the oracle finds by bisection (the
  mass-ratio root, the massive rescaling factor) against closed forms;
* the integrand's derivatives with respect to every coordinate of the unit
  point and the top mass against Richardson-extrapolated central differences
  of the oracle itself (which converge to the derivative independently of the
  dual arithmetic).
"""
import math

import numpy as np
import pytest

import workloads as W
from oracle import phasespace as ps
from oracle.dual import Dual


def _var(x):
    return Dual.variables([np.asarray(x, dtype=np.float64)])[0]


def test_elementary_rules():
    x = np.linspace(0.2, 3.0, 11)
    X = _var(x)
    cases = [(np.sqrt(X), 0.5 / np.sqrt(x)), (np.exp(X), np.exp(x)), (np.log(X), 1 / x),
             (np.sin(X), np.cos(x)), (np.cos(X), -np.sin(x)), (X ** 3, 3 * x ** 2), (1.0 / X, -1 / x ** 2),
             (X * X - 2.0 * X, 2 * x - 2), ((X + 1.0) / (X - 5.0), -6 / (x - 5) ** 2),
             (np.maximum(X, 1.0), (x >= 1.0) * 1.0)]
    for y, dy in cases:
        assert np.allclose(y.d[:, 0], dy, rtol=1e-14, atol=1e-15)
    # complex values and conjugation: d|z|^2/dx for z = (1 + 2i) x^2
    Z = (1 + 2j) * X * X
    m = np.real(np.einsum("n,n->n", np.conj(Z), Z))
    assert np.allclose(m.d[:, 0], 5 * 4 * x ** 3, rtol=1e-14)


def test_implicit_roots():
    # mass ratio: x(r) solves F(x) = 2x - x^2 = r (m = 2): dx/dr = 1/(2(1-x))
    r = np.array([0.1, 0.5, 0.9, 1 - 1e-9])
    x, d = ps._mass_ratio(_var(r), 2, complement=True)
    assert np.allclose(x.d[:, 0], 0.5 / np.sqrt(1 - r), rtol=1e-12)
    assert np.allclose(d.d[:, 0], -0.5 / np.sqrt(1 - r), rtol=1e-12)
    # two-body rescaling at sqrt(s), masses m1 = m2 = m: |k| = sqrt(s/4 - m^2),
    # so d|k|/dm = -m / |k| and the weight beta/(8 pi) has d/dm = -4 m /(s beta) / (8 pi)
    rs = np.array([400.0, 800.0, 2000.0])
    p = ps.massless_diet(np.random.default_rng(0).random((2, 3)), rs)
    M = _var(173.0)
    k, wfac, ok = ps.massive(p, [M, M], rs)
    kabs = np.sqrt(k.v[:, 0, 1] ** 2 + k.v[:, 0, 2] ** 2 + k.v[:, 0, 3] ** 2)
    dk = (k.d[:, 0, 1, 0] * k.v[:, 0, 1] + k.d[:, 0, 2, 0] * k.v[:, 0, 2] + k.d[:, 0, 3, 0] * k.v[:, 0, 3]) / kabs
    assert np.allclose(dk, -173.0 / kabs, rtol=1e-10)
    beta = np.sqrt(1 - 4 * 173.0 ** 2 / rs ** 2)
    w = ps.massless_weight(2, rs ** 2) * wfac
    assert np.allclose(w.d[:, 0], -4 * 173.0 / (rs ** 2 * beta) / (8 * math.pi), rtol=1e-10)


def _rich(fun, h):
    d1 = (fun(h) - fun(-h)) / (2 * h)
    d2 = (fun(h / 2) - fun(-h / 2)) / h
    return d2 + (d2 - d1) / 3


@pytest.mark.parametrize("name,n", [("ee_mumu", 8), ("gg_ttx", 8), ("uux_ttx", 8), ("gg_ttxg", 6), ("uux_ttxg", 6)])
def test_integrand_gradient_against_differences(oracle_processes, name, n):
    from oracle.integrand import Integrand
    wl = W.WORKLOADS[name]
    I = Integrand(wl, process=oracle_processes(name))
    x = np.clip(W.uniform_points(wl.ndim, n, 45), 1e-3, 1 - 1e-3)
    f, dx, dm = I.gradient(x)
    ref = I(x)
    nz = ref != 0
    assert np.max(np.abs(f[nz] / ref[nz] - 1)) < 1e-12
    for j in range(wl.ndim):
        def fx(h, j=j):
            xx = x.copy()
            xx[j] += h
            return I(xx)
        d = _rich(fx, 1e-4)
        err = np.abs(dx[j] - d)[nz] / (np.abs(d) + np.abs(ref))[nz]
        assert err.max() < 1e-8, (j, err.max())
    if wl.beams:
        mt = wl.m_top
        d = _rich(lambda h: Integrand(wl, m_top=mt + h)(x), 1e-3 * mt)
        err = np.abs(dm - d)[nz] / (np.abs(d) + np.abs(ref) / mt)[nz]
        assert err.max() < 1e-8, err.max()
