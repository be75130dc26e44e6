"""Phase space of the oracle (Sec. 2.4 of the MadFlow paper: a vectorised
RAMBO maps the integrator's random variables to flat phase space).

Definitions used here (all FP64, vectorised over events, momenta [N, n, 4] as
(E, px, py, pz), metric (+,-,-,-)):

* ``xmap``: parton momentum fractions from two unit numbers (the paper's
  L(x1, x2) of Fig. 1 has no stated map; reading: tau = tau_min^y1,
  x1 = tau^y2, x2 = tau / x1, Jacobian tau ln(1/tau_min) ln(1/tau)).
* ``massless_diet``: flat massless n-body phase space from 3n-4 unit numbers
  ("RAMBO on diet", S. Platzer, arXiv:1308.2922): a chain of two-body decays
  Q_k -> q_k + Q_{k+1}, with the squared-mass ratio x = M_{k+1}^2 / M_k^2 of a
  daughter system of m massless particles drawn from the density
  (1-x) x^(m-2) (CDF m x^(m-1) - (m-1) x^m) and isotropic decay angles.
  Per decay step k the unit numbers are (cos-theta, phi[, mass ratio]).
* ``massive``: the momentum rescaling of RAMBO (R. Kleiss, W.J. Stirling,
  S.D. Ellis, Comput. Phys. Commun. 40 (1986) 359): solve
  sum_i sqrt(m_i^2 + xi^2 |p_i|^2) = sqrt(s) for xi, rescale the 3-momenta,
  and multiply the massless weight by
  (sum|k|/sqrt s)^(2n-3) prod(|k_i|/k_i^0) sqrt(s) / sum(|k_i|^2/k_i^0).
* ``massless_weight``: (2 pi)^(4-3n) (pi/2)^(n-1) s^(n-2) / ((n-1)! (n-2)!).
* ``rambo_classic``: the original 4n-number massless RAMBO, kept only as an
  independent check of the flat measure.

The oracle finds xi by bisection to the last bit (the GPU path uses Newton):
the root is unique, so both must agree to rounding.
"""
from __future__ import annotations

import math

import numpy as np

from oracle.dual import Dual, as_f64, newton_root, value


def massless_weight(n: int, s):
    return ((2.0 * math.pi) ** (4 - 3 * n) * (math.pi / 2.0) ** (n - 1)
            * as_f64(s) ** (n - 2)
            / (math.factorial(n - 1) * math.factorial(n - 2)))


def xmap(y1, y2, tau_min: float):
    """(x1, x2, tau, jacobian) from two unit numbers."""
    if not value(tau_min) > 0.0:
        raise ValueError("the tau map needs a positive threshold")
    y1 = as_f64(y1)
    y2 = as_f64(y2)
    tau = np.exp(y1 * np.log(tau_min))
    x1 = np.exp(y2 * np.log(tau))
    x2 = tau / x1
    jac = tau * np.log(1.0 / tau_min) * np.log(1.0 / tau)
    return x1, x2, tau, jac


def _boost_from_rest(p, Q, M):
    """Boost p (given in the rest frame of Q, mass M) to the frame where Q is given."""
    p0 = p[..., 0]
    pv = p[..., 1:]
    Qv = Q[..., 1:]
    e = (Q[..., 0] * p0 + np.sum(Qv * pv, axis=-1)) / M
    c = (p0 + e) / (Q[..., 0] + M)
    out = np.empty_like(p)
    out[..., 0] = e
    out[..., 1:] = pv + c[..., None] * Qv
    return out


def _bisect(G, target, iters=200):
    """Root of the increasing function G on [0, 1] with G(root) = target."""
    lo = np.zeros_like(target)
    hi = np.ones_like(target)
    for _ in range(iters):
        mid = 0.5 * (lo + hi)
        below = G(mid) < target
        lo = np.where(below, mid, lo)
        hi = np.where(below, hi, mid)
    return 0.5 * (lo + hi)


def _mass_ratio(r, m: int, complement: bool = False):
    """Solve F(x) = m x^(m-1) - (m-1) x^m = r for x in [0, 1].

    For r <= 1/2 by bisection on F(x) = r.  For r > 1/2 the root is close to
    1, where F is flat and F(x) = r fixes 1 - x only to sqrt(eps); there the
    same equation is solved for d = 1 - x in the form 1 - F(1 - d) = 1 - r,
    with 1 - F(1 - d) = sum_{k>=2} c_k (-d)^k expanded with exact integer
    coefficients c_k = (m-1) C(m, k) - m C(m-1, k) (1 - r is exact for
    r >= 1/2).  With complement=True returns (x, d) with d = 1 - x carried
    to full relative precision (rounding x to a double near 1 would lose it).
    """
    if isinstance(r, Dual):
        # the root's value as for plain numbers, its tangent from the implicit
        # function theorem: dx = dr / F'(x), F'(x) = m (m-1) x^(m-2) (1 - x)
        xv, dv = _mass_ratio(r.v, m, complement=True)
        slope = m * (m - 1) * xv ** (m - 2) * dv
        dx = r.d / np.where(slope > 0, slope, np.inf)[..., None]
        x = Dual(xv, dx)
        return (x, Dual(dv, -dx)) if complement else x
    r = np.asarray(r, dtype=np.float64)
    low = _bisect(lambda x: m * x ** (m - 1) - (m - 1) * x ** m, r)
    coef = [(m - 1) * math.comb(m, k) - m * math.comb(m - 1, k) for k in range(m + 1)]
    G = lambda d: sum(coef[k] * (-d) ** k for k in range(2, m + 1))
    d_high = _bisect(G, 1.0 - r)
    x = np.where(r <= 0.5, low, 1.0 - d_high)
    if complement:
        return x, np.where(r <= 0.5, 1.0 - low, d_high)
    return x


def massless_diet(u, sqrt_s):
    """Flat massless momenta from unit numbers u [3n-4, N]; returns p [N, n, 4].

    Step k (k = 0 .. n-2) consumes (cos-theta, phi) and, for k <= n-3, the
    mass-ratio number, in that order.
    """
    u = as_f64(u)
    nr, N = u.shape
    n = (nr + 4) // 3
    if 3 * n - 4 != nr or n < 2:
        raise ValueError("need 3n-4 unit numbers with n >= 2")
    sqrt_s = np.broadcast_to(as_f64(sqrt_s), (N,))
    like = u if isinstance(u, Dual) else sqrt_s
    p = np.zeros((N, n, 4), like=like)
    Q = np.zeros((N, 4), like=like)
    Q[:, 0] = sqrt_s
    M = sqrt_s.copy()
    col = 0
    for k in range(n - 1):
        cth = 2.0 * u[col] - 1.0
        phi = 2.0 * math.pi * u[col + 1]
        col += 2
        m_daughter = n - k - 1            # massless particles left in Q_{k+1}
        if m_daughter >= 2:
            x, d = _mass_ratio(u[col], m_daughter, complement=True)
            col += 1
            M_next = M * np.sqrt(x)
        else:
            d = np.ones_like(M)
            M_next = np.zeros_like(M)
        # energy of the massless daughter in the rest frame of Q_k:
        # (M^2 - M_next^2) / (2M) = M (1 - x) / 2, taken from 1 - x directly
        e = 0.5 * M * d
        sth = np.sqrt(np.maximum(0.0, 1.0 - cth * cth))
        q = np.stack([e, e * sth * np.cos(phi), e * sth * np.sin(phi), e * cth], axis=-1)
        rest = np.stack([M - e, -q[:, 1], -q[:, 2], -q[:, 3]], axis=-1)
        p[:, k] = _boost_from_rest(q, Q, M)
        Qn = _boost_from_rest(rest, Q, M)
        if k == n - 2:
            p[:, n - 1] = Qn
        Q = Qn
        M = M_next
    return p


def massive(p, masses, sqrt_s):
    """Rescale massless momenta p [N, n, 4] (sum = (sqrt s, 0)) to the masses.

    Returns (k [N, n, 4], weight factor relative to the massless weight,
    ok mask).  Events below threshold get ok = False and zero weight.
    """
    p = as_f64(p)
    N, n, _ = p.shape
    m = np.stack(list(masses)) if any(isinstance(q, Dual) for q in masses) else np.asarray(masses, dtype=np.float64)
    sqrt_s = np.broadcast_to(as_f64(sqrt_s), (N,))
    ok = sqrt_s > np.sum(m)
    if np.all(m == 0.0):
        return p.copy(), np.ones(N), ok
    E = p[:, :, 0]
    mv, Ev, sv = value(m), value(E), value(sqrt_s)
    lo = np.zeros(N)
    hi = np.ones(N)
    for _ in range(200):
        mid = 0.5 * (lo + hi)
        F = np.sum(np.sqrt(mv[None, :] ** 2 + (mid[:, None] * Ev) ** 2), axis=1) - sv
        below = F < 0.0
        lo = np.where(below, mid, lo)
        hi = np.where(below, hi, mid)
    xi = 0.5 * (lo + hi)
    # dual inputs: the root's tangent by one Newton step in dual arithmetic
    xi = newton_root(lambda z: np.sum(np.sqrt(m[None, :] ** 2 + (z[:, None] * E) ** 2), axis=1) - sqrt_s,
                     lambda z: np.sum(z[:, None] * Ev ** 2 / np.sqrt(mv[None, :] ** 2 + (z[:, None] * Ev) ** 2),
                                      axis=1), xi)
    k = np.zeros(p.shape, like=xi) if isinstance(xi, Dual) else np.empty_like(p)
    k[:, :, 1:] = xi[:, None, None] * p[:, :, 1:]
    kabs = xi[:, None] * E
    k[:, :, 0] = np.sqrt(m[None, :] ** 2 + kabs ** 2)
    w = ((np.sum(kabs, axis=1) / sqrt_s) ** (2 * n - 3)
         * np.prod(kabs / k[:, :, 0], axis=1)
         * sqrt_s / np.sum(kabs ** 2 / k[:, :, 0], axis=1))
    w = np.where(ok, w, 0.0)
    return k, w, ok


def rambo_classic(u, sqrt_s, n: int):
    """Original massless RAMBO from 4n unit numbers u [4n, N]."""
    u = np.asarray(u, dtype=np.float64)
    N = u.shape[1]
    q = np.zeros((N, n, 4))
    for i in range(n):
        c = 2.0 * u[4 * i] - 1.0
        phi = 2.0 * math.pi * u[4 * i + 1]
        q0 = -np.log(u[4 * i + 2] * u[4 * i + 3])
        s = np.sqrt(1.0 - c * c)
        q[:, i] = np.stack([q0, q0 * s * np.cos(phi), q0 * s * np.sin(phi), q0 * c], axis=-1)
    Qs = q.sum(axis=1)
    M = np.sqrt(Qs[:, 0] ** 2 - np.sum(Qs[:, 1:] ** 2, axis=1))
    b = -Qs[:, 1:] / M[:, None]
    x = sqrt_s / M
    gamma = Qs[:, 0] / M
    a = 1.0 / (1.0 + gamma)
    p = np.zeros_like(q)
    for i in range(n):
        bq = np.sum(b * q[:, i, 1:], axis=1)
        p[:, i, 0] = x * (gamma * q[:, i, 0] + bq)
        p[:, i, 1:] = x[:, None] * (q[:, i, 1:] + b * q[:, i, 0:1] + (a * bq)[:, None] * b)
    return p
