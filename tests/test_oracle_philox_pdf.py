"""Pins of the oracle's random numbers and PDF interpolation (CPU only)."""
import math

import numpy as np
import pytest

import workloads as W
from oracle import philox
from oracle.pdf import PdfTable, xfx_scalar


# ----------------------------------------------------------------- Philox
def test_philox_matches_numpy_library():
    # numpy's Philox bit generator is an independent Philox4x64-10; its first
    # block is generated at counter + 1.
    rng = np.random.Generator(np.random.PCG64(7))
    for _ in range(20):
        key = rng.integers(0, 2 ** 63, size=2, dtype=np.uint64) * np.uint64(2) + np.uint64(1)
        ctr = rng.integers(0, 2 ** 63, size=4, dtype=np.uint64)
        bg = np.random.Philox(key=key, counter=ctr)
        ref = bg.random_raw(8)
        c1 = ctr.copy(); c1[0] += np.uint64(1)
        c2 = ctr.copy(); c2[0] += np.uint64(2)
        mine = philox.philox4x64_10(np.stack([c1, c2]), key).ravel()
        assert np.array_equal(mine, ref)


def test_philox_counter_carry_matches_numpy():
    key = np.array([3, 5], dtype=np.uint64)
    ctr = np.array([2 ** 64 - 1, 2 ** 64 - 1, 9, 0], dtype=np.uint64)
    ref = np.random.Philox(key=key, counter=ctr).random_raw(4)
    mine = philox.philox4x64_10(np.array([[0, 0, 10, 0]], dtype=np.uint64), key).ravel()
    assert np.array_equal(mine, ref)


def test_unit_conversion_is_open_interval_and_exact():
    r = np.array([0, 1, 2 ** 11, 2 ** 64 - 1], dtype=np.uint64)
    u = philox.to_unit(r)
    assert u[0] == 2.0 ** -53 and u[1] == 2.0 ** -53
    assert u[3] == 1.0 - 2.0 ** -53
    assert np.all((u > 0) & (u < 1))


def test_vegas_uniforms_layout_and_moments():
    u = philox.vegas_uniforms(seed=11, iteration=2, subprocess=1, first_event=5, n=20000, ndim=7)
    assert u.shape == (7, 20000)
    # dimension j of event e is word j % 4 of the block j // 4
    key = np.array([11, 0], dtype=np.uint64)
    w = philox.philox4x64_10(np.array([[5 + 3, 2, 1, 1]], dtype=np.uint64), key)[0]
    assert u[6, 3] == philox.to_unit(w[2:3])[0]
    # uniform moments within 5 standard errors
    n = u.shape[1]
    assert np.all(np.abs(u.mean(axis=1) - 0.5) < 5 * math.sqrt(1 / 12 / n))
    assert np.all(np.abs((u ** 2).mean(axis=1) - 1 / 3) < 5 * math.sqrt(4 / 45 / n))
    # different iterations give different streams
    v = philox.vegas_uniforms(seed=11, iteration=3, subprocess=1, first_event=5, n=100, ndim=7)
    assert not np.any(v == u[:, :100])


# ----------------------------------------------------------------- PDF
def _table_from(fun):
    xs, qs = W.x_knots(), W.q2_knots()
    a, b = np.log(xs), np.log(qs)
    v = fun(a[None, :], b[:, None])
    return PdfTable(v, W.PDF_X_MIN, W.PDF_X_MAX, W.PDF_Q2_MIN, W.PDF_Q2_MAX)


def test_pdf_exact_at_knots():
    tab = PdfTable(W.pdf_table("g", q2_slope=0.1), W.PDF_X_MIN, W.PDF_X_MAX, W.PDF_Q2_MIN, W.PDF_Q2_MAX)
    xs, qs = W.x_knots(), W.q2_knots()
    rng = np.random.default_rng(3)
    i = rng.integers(0, W.PDF_NX - 1, 300)
    j = rng.integers(0, W.PDF_NQ - 1, 300)
    got = tab.xfx(xs[i], qs[j])
    ref = tab.v[j, i]
    assert np.allclose(got, ref, rtol=1e-13, atol=1e-300)


def test_pdf_biquadratic_exact_on_interior_intervals():
    fun = lambda a, b: 1.5 + 0.3 * a - 0.2 * a * a + 0.05 * b + 0.01 * a * b - 0.003 * b * b \
        + 0.002 * a * a * b * b
    tab = _table_from(fun)
    rng = np.random.default_rng(4)
    # interior intervals: i in [1, nx-3], j in [1, nq-3]
    ai = rng.uniform(tab.a[1], tab.a[-2], 500)
    bj = rng.uniform(tab.b[1], tab.b[-2], 500)
    got = tab.xfx(np.exp(ai), np.exp(bj))
    assert np.max(np.abs(got - fun(ai, bj))) < 1e-12


def test_pdf_bilinear_exact_everywhere():
    fun = lambda a, b: 2.0 + 0.7 * a - 0.05 * b + 0.01 * a * b
    tab = _table_from(fun)
    rng = np.random.default_rng(5)
    ai = rng.uniform(tab.a[0], tab.a[-1], 500)
    bj = rng.uniform(tab.b[0], tab.b[-1], 500)
    got = tab.xfx(np.exp(ai), np.exp(bj))
    assert np.max(np.abs(got - fun(ai, bj))) < 1e-12


def test_pdf_vectorised_equals_scalar_definition():
    tab = PdfTable(W.pdf_table("u", q2_slope=0.1), W.PDF_X_MIN, W.PDF_X_MAX, W.PDF_Q2_MIN, W.PDF_Q2_MAX)
    rng = np.random.default_rng(6)
    xs = np.exp(rng.uniform(math.log(1e-6), 0, 200))
    qs = np.exp(rng.uniform(0, math.log(1e8), 200))
    qs[:3] = [1.0, 1.0001, 0.99e8]
    vec = tab.xfx(xs, qs)
    sca = np.array([xfx_scalar(tab, x, q) for x, q in zip(xs, qs)])
    assert np.allclose(vec, sca, rtol=1e-14, atol=1e-300)


def test_pdf_close_to_analytic_gluon():
    tab = PdfTable(W.pdf_table("g"), W.PDF_X_MIN, W.PDF_X_MAX, W.PDF_Q2_MIN, W.PDF_Q2_MAX)
    xs = np.exp(np.linspace(math.log(7e-4), math.log(0.6), 400))
    got = tab.xfx(xs, W.M_TOP ** 2)
    ref = W.xg_analytic(xs)
    # cubic Hermite with difference slopes: the slope error is O(h^2) times
    # the third derivative in ln x (h = ln(1e6)/99); it grows with (1-x)^5's
    # curvature towards large x.  An index or slope bug gives O(1) errors.
    rel = np.abs(got / ref - 1)
    assert np.max(rel[xs < 1e-2]) < 1e-5
    assert np.max(rel) < 5e-3


def test_pdf_normalisations():
    from scipy.integrate import quad
    mom, _ = quad(lambda x: float(W.xg_analytic(x)), 0, 1, limit=200)
    num, _ = quad(lambda x: float(W.xu_analytic(x)) / x, 0, 1, limit=200)
    assert abs(mom - 0.5) < 1e-9
    assert abs(num - 2.0) < 1e-9
