"""Weighted histograms of observables of a Vegas pass (the differential
distributions of Sec. 3.1 of the MadFlow paper: the transverse momentum and
pseudorapidity of the top quark, Fig. 2).  Test infrastructure only.

Definitions, for a final-state leg with collider-frame momentum (E, px, py, pz)
(the partonic centre-of-mass momenta boosted along the beam axis by the
rapidity of the parton pair, as for event records):

* transverse momentum   pT  = sqrt(px^2 + py^2);
* rapidity              y   = (1/2) ln((E + pz) / (E - pz));
* pseudorapidity        eta = asinh(pz / pT).

An observable with nbins equal bins on [lo, hi) puts a value v in bin
b = floor((v - lo) * s), s = nbins / (hi - lo) evaluated once in FP64; values
with b outside 0 .. nbins-1 are not binned, nor are points that fail the
threshold or the cuts.  For N points with weights w_i = f(x_i) J_V(y_i):

* sigma_b = (1/N) sum_{i in b} w_i                 (pb in the bin),
* err_b   = sqrt((sum_{i in b} w_i^2 / N - sigma_b^2) / (N - 1)),
* count_b = number of points in the bin.

(sum_b sigma_b over a range that holds every point is the pass's integral
estimate; err_b is the Monte Carlo error of sigma_b.)
"""
from __future__ import annotations

import numpy as np

PT, RAPIDITY, PSEUDORAPIDITY = 0, 1, 2


def values(p_lab: np.ndarray, kind: int, leg: int) -> np.ndarray:
    """Observable `kind` of leg `leg` for momenta p_lab [N, n, 4] (E, px, py, pz)."""
    E, px, py, pz = (p_lab[:, leg, q] for q in range(4))
    pt = np.hypot(px, py)
    if kind == PT:
        return pt
    if kind == RAPIDITY:
        return 0.5 * np.log((E + pz) / (E - pz))
    if kind == PSEUDORAPIDITY:
        return np.arcsinh(pz / pt)
    raise ValueError("unknown observable")


def bin_index(v: np.ndarray, nbins: int, lo: float, hi: float) -> np.ndarray:
    """Bin of each value, -1 outside [lo, hi)."""
    s = nbins / (hi - lo)
    t = (v - lo) * s
    b = np.floor(t)
    inside = (t >= 0) & (b < nbins)
    return np.where(inside, b, -1).astype(np.int64)


def histogram(w: np.ndarray, b: np.ndarray, nbins: int, n_points: int):
    """(sigma, err, count) per bin from weights w and bins b (-1: not binned)."""
    sigma = np.zeros(nbins)
    sq = np.zeros(nbins)
    count = np.zeros(nbins, dtype=np.int64)
    for k in range(nbins):
        sel = b == k
        sigma[k] = np.sum(w[sel]) / n_points
        sq[k] = np.sum(w[sel] ** 2) / n_points
        count[k] = int(np.count_nonzero(sel))
    var = (sq - sigma ** 2) / (n_points - 1)
    return sigma, np.sqrt(np.maximum(var, 0.0)), count


def histograms(p_lab: np.ndarray, passing: np.ndarray, w: np.ndarray, observables):
    """One (sigma, err, count) per observable (kind, leg, nbins, lo, hi) for the
    points of a pass: momenta p_lab [N, n, 4], passing [N] (threshold and cuts),
    weights w [N]."""
    n = w.shape[0]
    out = []
    for kind, leg, nbins, lo, hi in observables:
        b = bin_index(values(p_lab, kind, leg), nbins, lo, hi)
        b = np.where(passing, b, -1)
        out.append(histogram(w, b, nbins, n))
    return out
