"""Pins of the oracle's unweighting and event frame (CPU only)."""
import numpy as np
import pytest

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
