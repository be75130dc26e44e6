"""Topology-aware multichannel phase space (oracle).  TEST INFRASTRUCTURE:
only tests/, the smoke check and the bench's CPU-baseline leg use this module.

The paper's phase space is flat (RAMBO, Sec. 2.4) and it names the cost of
that choice: many points for high multiplicities and about 5 % unweighting
efficiency (Sec. 2.5, Sec. 2.6 "Scope"); its outlook (Sec. 4) is a phase
space built from the process topology, with multichannel weight
optimisation (Kleiss & Pittau, ref. [Kleiss:1994qy]) as the recommended
route.  This module is the plain definition of the multichannel method the
library implements; every reading below is ours (the paper gives none).

Channels.  Every tree diagram of the process without a four-gluon vertex
gives a channel; diagrams with the same channel are merged.  A diagram's
propagators split into
  * t-channel propagators: those on the path between the incoming legs a
    (leg 0, along +z) and b (leg 1); their final-state legs on a's side form
    nested sets F_1 < F_2 < ... < F_{k-1};
  * s-channel propagators: all others; each carries a cluster X of final
    legs (for a propagator whose far side holds both a and b: the final legs
    of its near side).
The maximal clusters c_j = F_j \\ F_{j-1} (F_0 = {}, F_k = all final legs)
are attached to the spine in that order; each is one leg or an s-cluster.
Inside an s-cluster the propagators form a binary tree (left child: the part
holding the smallest final index).  With no t-channel propagator (k = 1)
the whole final state is one s-cluster whose invariant mass is s-hat.

Mapping of the 3n-4 unit numbers u (n final particles), in this order:
  (i)   for j = 1..k with |c_j| >= 2: s_{c_j} in
        [m(c_j)^2, (sqrt(s-hat) - sum_{i<j} sqrt(s_{c_i}) - sum_{i>j} m(c_i))^2]
        (m(X) = sum of the final masses in X; a single leg has s = m^2);
  (ii)  for j = 1..k-2: the remainder R_j = c_{j+1} + ... + c_k, s_{R_j} in
        [(sum_{i>j} sqrt(s_{c_i}))^2, (sqrt(s_{R_{j-1}}) - sqrt(s_{c_j}))^2],
        flat (R_0 is the whole final state, s = s-hat; R_{k-1} = c_k);
  (iii) for j = 1..k-1, the split R_{j-1} -> c_j + R_j: in the rest frame of
        R_{j-1}, c_j's polar angle about the direction of
        q_{j-1} = p_a - c_1 - ... - c_{j-1} takes the density of the
        t-channel propagator, prop. to 1 / (M_j^2 + t0 - t_j) in
        t_j = (q_{j-1} - c_j)^2 (one number), and its azimuth about that axis
        is flat (one number; the axis frame is R_z(phi_q) R_y(theta_q) of
        the axis' polar and azimuthal angles);
  (iv)  for each maximal cluster in spine order, its nodes X -> (L, R) in
        pre-order: s_L (if L is a cluster) in [m(L)^2, (sqrt(s_X) - m(R))^2],
        s_R (if R is a cluster) in [m(R)^2, (sqrt(s_X) - sqrt(s_L))^2], then
        L's direction in the rest frame of X, isotropic (cos theta, phi
        about the fixed axes).
An s-cluster's mass takes the density of its propagator,
prop. to 1 / (s - M^2 + s0) on its range (flat where lo - M^2 + s0 <= 0);
two-body momenta are built in the parent's rest frame and boosted to the
partonic centre-of-mass frame without rotation.

Weight.  With dPhi_n = prod ds/(2 pi) prod dPhi_2 and
dPhi_2 = lambda^(1/2)(s; s_1, s_2) / (32 pi^2 s) dOmega (the convention of
the RAMBO weight of Sec. 2.4), the channel's density g_i is the product of
its sampling densities divided by these factors.  The integrand is split as
f = sum_i a_i f with the partition a_i = P_i / sum_j P_j, where P_i is the
product over channel i's propagators of 1 / (|x - M^2| + r)^2 (x = s of an
s-cluster, including s-hat for k = 1, or t_j; r = s0 or t0) -- the
single-diagram-enhanced split with the diagram's propagator structure in
place of its |amplitude|^2.  Channel i integrates f a_i / g_i over its own
unit hypercube with its own Vegas grid; the cross section is the sum of
the channel integrals and its variance the sum of theirs.

Allocation.  The points of an iteration are shared out by Neyman's rule for
a sum of independent estimates: n_i = n_floor + floor(F sigma_i / sum_j
sigma_j), F = N - K n_floor, sigma_i the per-point standard deviation of
channel i's weights (equal shares when every sigma_i is zero).  A deviation
estimated from few points is unreliable (a channel whose few points missed
its peak would be starved), so it is first shrunk towards the pooled one as
if m0 more points had shown the pooled variance.
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np

from . import phasespace as ps
from .feynman import Process

TWO_PI = 2.0 * math.pi


# ----------------------------------------------------------------------------
# channels from the diagrams
# ----------------------------------------------------------------------------
@dataclass(frozen=True)
class Cluster:
    """An s-channel propagator over the final-state indices in `legs`
    (0-based among the final particles), with its two children (a Cluster
    or a final index)."""
    legs: frozenset
    mass: int            # mass id of the propagator: 0 = top, -1 = massless
    left: object
    right: object


@dataclass(frozen=True)
class Channel:
    spine: tuple         # c_1 .. c_k: Cluster or final index
    t_mass: tuple        # mass ids of the k-1 t-channel propagators
    root_mass: int       # k = 1: mass id of the propagator into the final state
    key: tuple

    @property
    def k(self):
        return len(self.spine)


def _legs(x):
    return x.legs if isinstance(x, Cluster) else frozenset((x,))


def _mask(legs):
    return sum(1 << i for i in legs)


def _mass_id(line):
    # a propagator's flavour: the top quark is mass 0, everything else massless
    return 0 if (line[0] == "F" and line[1] == "t") else -1


def _edges(tree):
    """(leg set over all legs, mass id, kind) of every node below the top of
    an oracle diagram tree (the top node's line is the last external leg)."""
    out = []

    def walk(node, top):
        if node[0] == "L":
            return
        _, kind, line, children, _ = node
        if not top:
            out.append((frozenset(Process.legs_of(node)), _mass_id(line), kind))
        for c in children:
            walk(c, False)
    walk(tree, True)
    return out


def _has_four_vertex(tree):
    if tree[0] == "L":
        return False
    return tree[1] == "vvvv" or any(_has_four_vertex(c) for c in tree[3])


def _cluster_tree(S, s_masses):
    """The binary tree of s-clusters inside the final-index set S."""
    inner = [X for X in s_masses if X < S]
    maximal = [X for X in inner if not any(X < Y for Y in inner)]
    covered = frozenset().union(*maximal) if maximal else frozenset()
    parts = list(maximal) + [frozenset((i,)) for i in sorted(S - covered)]
    if len(parts) != 2:
        raise ValueError("an s-channel node without exactly two children")
    parts.sort(key=min)
    kids = [(_cluster_tree(P, s_masses) if len(P) >= 2 else min(P)) for P in parts]
    return Cluster(S, s_masses[S], kids[0], kids[1])


def _key(spine, t_mass, s_masses):
    cm = [_mask(_legs(c)) for c in spine]
    sl = sorted((_mask(X), m) for X, m in s_masses.items())
    return tuple([len(spine)] + cm + list(t_mass) + [len(sl)] + [v for pair in sl for v in pair])


def derive_channels(proc: Process):
    """The channels of an oracle process, merged and in ascending key order.
    The key is (k, masks of c_1..c_k, t-channel mass ids, number of
    s-clusters, their (mask, mass id) pairs in ascending order); masks have
    bit i for final index i."""
    n = proc.n
    finals = frozenset(range(n - 2))
    found = {}
    for tree in proc.diagrams:
        if _has_four_vertex(tree):
            continue
        s_masses, t_edges, root_mass = {}, {}, -1
        for S, m, _ in _edges(tree):
            has_a, has_b = 0 in S, 1 in S
            fin = frozenset(i - 2 for i in S if i >= 2)
            if not has_a and not has_b:
                s_masses[fin] = m
            elif has_a and has_b:
                X = finals - fin
                s_masses[X] = m
                if X == finals:
                    root_mass = m
            else:
                side = fin if has_a else finals - fin
                t_edges[side] = m
        F = sorted(t_edges, key=len)
        bounds = [frozenset()] + F + [finals]
        spine = []
        for j in range(1, len(bounds)):
            c = bounds[j] - bounds[j - 1]
            if not bounds[j - 1] < bounds[j]:
                raise ValueError("t-channel sets are not nested")
            spine.append(_cluster_tree(c, s_masses) if len(c) >= 2 else min(c))
        t_mass = tuple(t_edges[X] for X in F)
        key = _key(spine, t_mass, s_masses)
        found[key] = Channel(tuple(spine), t_mass, root_mass if not F else -1, key)
    return [found[k] for k in sorted(found)]


# ----------------------------------------------------------------------------
# kinematics helpers (vectorised over points; plain arrays or the dual numbers
# of oracle/dual.py, for derivatives)
# ----------------------------------------------------------------------------
def _total(xs):
    """Sum of a list of numbers or dual numbers (0 when empty)."""
    out = 0.0
    for x in xs:
        out = x + out
    return out


def _clip1(c):
    return np.minimum(np.maximum(c, -1.0), 1.0)
def _mdot(a, b):
    return a[..., 0] * b[..., 0] - a[..., 1] * b[..., 1] - a[..., 2] * b[..., 2] - a[..., 3] * b[..., 3]


def _sqrt_lambda(s, s1, s2):
    """lambda^(1/2)(s, s1, s2) as sqrt((s - (m1+m2)^2)(s - (m1-m2)^2))."""
    m1, m2 = np.sqrt(s1), np.sqrt(s2)
    a = np.maximum(s - (m1 + m2) ** 2, 0.0)
    b = np.maximum(s - (m1 - m2) ** 2, 0.0)
    return np.sqrt(a * b)


def _boost_to_rest(p, Q, M):
    """p given in the frame of Q (mass M) -> p in the rest frame of Q."""
    e = (Q[..., 0] * p[..., 0] - np.sum(Q[..., 1:] * p[..., 1:], axis=-1)) / M
    c = (p[..., 0] + e) / (Q[..., 0] + M)
    out = np.empty_like(p)
    out[..., 0] = e
    out[..., 1:] = p[..., 1:] - c[..., None] * Q[..., 1:]
    return out


def _mass_sample(u, lo, hi, M2, reg):
    """s in [lo, hi] with density prop. to 1/(s - M2 + reg) (flat where
    lo - M2 + reg <= 0) -> (s, 1/density)."""
    a = lo - M2 + reg
    pole = a > 0.0
    a_safe = np.where(pole, a, 1.0)
    L = np.log1p(np.where(pole, (hi - lo) / a_safe, 0.0))
    s_pole = lo + a_safe * np.expm1(u * L)
    inv_pole = (a_safe * np.exp(u * L)) * L
    s = np.where(pole, s_pole, lo + u * (hi - lo))
    inv = np.where(pole, inv_pole, hi - lo)
    return s, inv


def _mass_density_inv(s, lo, hi, M2, reg):
    """1/density of _mass_sample at s (for checks)."""
    a = lo - M2 + reg
    pole = a > 0.0
    L = np.log1p(np.where(pole, (hi - lo) / np.where(pole, a, 1.0), 0.0))
    return np.where(pole, (s - M2 + reg) * L, hi - lo)


def _direction(c, phi):
    st = np.sqrt(np.maximum((1.0 - c) * (1.0 + c), 0.0))
    return np.stack([st * np.cos(phi), st * np.sin(phi), c], axis=-1)


def _two_body(X, sX, sL, sR, n):
    """Momenta (frame of X) of daughters with masses^2 sL, sR, L along the
    unit vector n in the rest frame of X; and lambda^(1/2)."""
    M = np.sqrt(sX)
    lam = _sqrt_lambda(sX, sL, sR)
    p = lam / (2.0 * M)
    L = np.concatenate([((sX + sL - sR) / (2.0 * M))[..., None], p[..., None] * n], axis=-1)
    R = np.concatenate([((sX + sR - sL) / (2.0 * M))[..., None], -p[..., None] * n], axis=-1)
    return ps._boost_from_rest(L, X, M), ps._boost_from_rest(R, X, M), lam


# ----------------------------------------------------------------------------
# generation
# ----------------------------------------------------------------------------
def generate(ch: Channel, u, rs, fm, s0: float, t0: float, masses):
    """Final-state momenta [N, n, 4] (partonic CM frame), 1/g_i [N] and a
    validity flag [N] from unit numbers u [3n-4, N] through channel ch.
    fm: final masses [n]; masses: mass ids -> GeV (masses[0] = m_t)."""
    from .dual import Dual, as_f64
    u = as_f64(u)
    rs = as_f64(rs)
    N = u.shape[1]
    nf = len(fm)
    if not any(isinstance(v, Dual) for v in fm):
        fm = np.asarray(fm, dtype=np.float64)
    s_hat = rs * rs
    like = next((v for v in (u, rs) if isinstance(v, Dual)), None)
    p = np.zeros((N, nf, 4), like=like) if like is not None else np.zeros((N, nf, 4))
    inv_g = 1.0 + 0.0 * rs
    ok = np.ones(N, dtype=bool)
    col = [0]

    def take():
        v = u[col[0]]
        col[0] += 1
        return v

    def M2(mid):
        return 0.0 if mid < 0 else masses[mid] ** 2

    def mmin(x):
        return _total([fm[i] for i in sorted(_legs(x))])

    def const(v):
        return v + 0.0 * rs

    def mass_step(lo, hi, M2v, reg):
        nonlocal ok
        ok = ok & (hi >= lo)
        hi_c = np.maximum(hi, lo)
        s, inv = _mass_sample(take(), lo, hi_c, M2v, reg)
        return s, inv

    k = ch.k
    spine = ch.spine
    s_c = [None] * k
    # (i) maximal clusters
    for j in range(k):
        c = spine[j]
        if not isinstance(c, Cluster):
            s_c[j] = const(fm[c] ** 2)
            continue
        if k == 1:
            s_c[j] = s_hat
            continue
        top = rs - _total([np.sqrt(s_c[i]) for i in range(j)]) - _total([mmin(spine[i]) for i in range(j + 1, k)])
        lo = const(mmin(c) ** 2)
        s, inv = mass_step(lo, np.maximum(top, 0.0) ** 2, M2(c.mass), s0)
        s_c[j] = s
        inv_g = inv_g * inv / TWO_PI
    # (ii) chain remainders
    s_R = [s_hat] + [None] * max(k - 1, 0)
    if k >= 2:
        s_R[k - 1] = s_c[k - 1]
    for j in range(1, k - 1):
        lo = _total([np.sqrt(s_c[i]) for i in range(j, k)]) ** 2
        hi = np.maximum(np.sqrt(s_R[j - 1]) - np.sqrt(s_c[j - 1]), 0.0) ** 2
        ok = ok & (hi >= lo)
        hi = np.maximum(hi, lo)
        s_R[j] = lo + take() * (hi - lo)
        inv_g = inv_g * (hi - lo) / TWO_PI
    # (iii) the chain
    mom = [None] * k
    zero = np.zeros(N)
    R_prev = np.stack([rs, zero, zero, zero], axis=-1)
    q = np.stack([0.5 * rs, zero, zero, 0.5 * rs], axis=-1)
    for j in range(1, k):
        sRp = s_R[j - 1]
        sc = s_c[j - 1]
        sRj = s_R[j]
        Mr = np.sqrt(sRp)
        qs = _boost_to_rest(q, R_prev, Mr)
        qabs = np.sqrt(qs[:, 1] ** 2 + qs[:, 2] ** 2 + qs[:, 3] ** 2)
        q2 = _mdot(q, q)
        Ec = (sRp + sc - sRj) / (2.0 * Mr)
        lam = _sqrt_lambda(sRp, sc, sRj)
        pc = lam / (2.0 * Mr)
        A = M2(ch.t_mass[j - 1]) + t0 - q2 - sc + 2.0 * qs[:, 0] * Ec
        B = 2.0 * qabs * pc
        pole = (B > 0.0) & (A - B > 0.0)
        Bs = np.where(pole, B, 1.0)
        AmB = np.where(pole, A - B, 1.0)
        L = np.log1p(2.0 * Bs / AmB)
        uc = take()
        c_pole = -1.0 - (A + Bs) * np.expm1(-uc * L) / Bs
        cth = _clip1(np.where(pole, c_pole, 2.0 * uc - 1.0))
        inv_h = np.where(pole, (A - Bs * cth) * L / Bs, 2.0)
        phi = TWO_PI * take()
        # axis frame: R_z(phi_q) R_y(theta_q)
        qabs_s = np.where(qabs > 0.0, qabs, 1.0)
        hx = np.where(qabs > 0.0, qs[:, 1] / qabs_s, 0.0)
        hy = np.where(qabs > 0.0, qs[:, 2] / qabs_s, 0.0)
        hz = np.where(qabs > 0.0, qs[:, 3] / qabs_s, 1.0)
        rho = np.sqrt(hx * hx + hy * hy)
        rho_s = np.where(rho > 0.0, rho, 1.0)
        cphi_q = np.where(rho > 0.0, hx / rho_s, 1.0)
        sphi_q = np.where(rho > 0.0, hy / rho_s, 0.0)
        nl = _direction(cth, phi)
        vx = hz * nl[:, 0] + rho * nl[:, 2]
        vy = nl[:, 1]
        vz = -rho * nl[:, 0] + hz * nl[:, 2]
        n_dir = np.stack([cphi_q * vx - sphi_q * vy, sphi_q * vx + cphi_q * vy, vz], axis=-1)
        cj, Rj, lam2 = _two_body(R_prev, sRp, sc, sRj, n_dir)
        inv_g = inv_g * lam2 / (32.0 * math.pi ** 2 * sRp) * TWO_PI * inv_h
        mom[j - 1] = cj
        q = q - cj
        R_prev = Rj
    mom[k - 1] = R_prev

    # (iv) inside the clusters
    def split(node, X, sX):
        nonlocal inv_g, ok
        L, R = node.left, node.right
        if isinstance(L, Cluster):
            lo = const(mmin(L) ** 2)
            hi = np.maximum(np.sqrt(sX) - mmin(R), 0.0) ** 2
            sL, inv = mass_step(lo, hi, M2(L.mass), s0)
            inv_g = inv_g * inv / TWO_PI
        else:
            sL = const(fm[L] ** 2)
        if isinstance(R, Cluster):
            lo = const(mmin(R) ** 2)
            hi = np.maximum(np.sqrt(sX) - np.sqrt(sL), 0.0) ** 2
            sR, inv = mass_step(lo, hi, M2(R.mass), s0)
            inv_g = inv_g * inv / TWO_PI
        else:
            sR = const(fm[R] ** 2)
        cth = 2.0 * take() - 1.0
        phi = TWO_PI * take()
        PL, PR, lam = _two_body(X, sX, sL, sR, _direction(cth, phi))
        inv_g = inv_g * lam / (32.0 * math.pi ** 2 * sX) * (4.0 * math.pi)
        for child, P, s in ((L, PL, sL), (R, PR, sR)):
            if isinstance(child, Cluster):
                split(child, P, s)
            else:
                p[:, child] = P

    for j in range(k):
        c = spine[j]
        if isinstance(c, Cluster):
            split(c, mom[j], s_c[j])
        else:
            p[:, c] = mom[j]
    assert col[0] == u.shape[0], "unit numbers left over"
    return p, inv_g, ok


def n_units(ch: Channel) -> int:
    """Unit numbers the channel consumes (3n-4 for n final particles)."""
    nf = sum(len(_legs(c)) for c in ch.spine)
    return 3 * nf - 4


# ----------------------------------------------------------------------------
# partition
# ----------------------------------------------------------------------------
def _clusters(x):
    if isinstance(x, Cluster):
        yield x
        yield from _clusters(x.left)
        yield from _clusters(x.right)


def propagator_products(channels, pa, p, s0: float, t0: float, masses):
    """P_i [N, K]: the product over channel i's propagators of
    1 / (|x - M^2| + r)^2, at final momenta p [N, n, 4] and incoming a
    momentum pa [N, 4]."""
    N = p.shape[0]
    cols = []

    def M2(mid):
        return 0.0 if mid < 0 else masses[mid] ** 2

    def inv(x, m2, r):
        d = np.abs(x - m2) + r
        return 1.0 / (d * d)

    for i, ch in enumerate(channels):
        P = 1.0
        for c in ch.spine:
            for X in _clusters(c):
                if ch.k == 1 and X is c:
                    s = _mdot(np.sum(p[:, sorted(X.legs)], axis=1), np.sum(p[:, sorted(X.legs)], axis=1))
                    P = P * inv(s, M2(ch.root_mass), s0)
                    continue
                Q = np.sum(p[:, sorted(X.legs)], axis=1)
                P = P * inv(_mdot(Q, Q), M2(X.mass), s0)
        q = pa.copy()
        for j in range(ch.k - 1):
            q = q - np.sum(p[:, sorted(_legs(ch.spine[j]))], axis=1)
            P = P * inv(_mdot(q, q), M2(ch.t_mass[j]), t0)
        cols.append(P + 0.0 * pa[:, 0])
    return np.stack(cols, axis=1)


def partition(channels, pa, p, s0, t0, masses):
    """a_i [N, K] = P_i / sum_j P_j."""
    P = propagator_products(channels, pa, p, s0, t0, masses)
    return P / np.sum(P, axis=1)[:, None]


# ----------------------------------------------------------------------------
# allocation
# ----------------------------------------------------------------------------
def shrink(sigma, n_prev, m0: float):
    """Per-point standard deviations estimated from n_prev[k] points each,
    shrunk towards the pooled one as if m0 more points had shown the pooled
    variance: sqrt((n_k s_k^2 + m0 s^2) / (n_k + m0)), s^2 = sum_k n_k s_k^2 /
    sum_k n_k (sums in channel order)."""
    num, den = 0.0, 0.0
    for s_, n_ in zip(sigma, n_prev):
        num += float(n_) * float(s_) * float(s_)
        den += float(n_)
    pooled = num / den if den > 0.0 else 0.0
    return [math.sqrt((float(n_) * float(s_) * float(s_) + m0 * pooled) / (float(n_) + m0)) if float(n_) + m0 > 0.0
            else 0.0 for s_, n_ in zip(sigma, n_prev)]


def allocate(sigma, n_total: int, n_floor: int, n_prev=None, m0: float = 0.0):
    """Neyman allocation of n_total points over channels with per-point
    standard deviations sigma (every channel keeps n_floor); with n_prev, the
    deviations are first shrunk (shrink) with m0 pseudo-points."""
    sigma = [float(s) for s in sigma]
    if n_prev is not None:
        sigma = shrink(sigma, n_prev, float(m0))
    K = len(sigma)
    free = n_total - K * n_floor
    if free < 0:
        raise ValueError("fewer points than the floors need")
    S = 0.0
    for s in sigma:
        S += s
    if not S > 0.0:
        return [n_floor + free // K for _ in range(K)]
    return [n_floor + int(math.floor(float(free) * (s / S))) for s in sigma]
