"""Vegas adaptive importance sampling (oracle).

The paper integrates with VegasFlow (Sec. 1, Sec. 2.2) and does not restate
the algorithm; this oracle follows G.P. Lepage, J. Comput. Phys. 27 (1978)
192, in the per-dimension grid form:

* grid: for each dimension j, N_b + 1 increasing edges e_j0 = 0 < ... <
  e_jN_b = 1;
* map:  for a unit number y, bin i = floor(y N_b), x = e_i + (y N_b - i)
  (e_{i+1} - e_i), Jacobian N_b (e_{i+1} - e_i); the point's weight is
  w = f(x) prod_j J_j;
* one iteration of N points: I = sum w / N, variance of I =
  (sum w^2 / N - I^2) / (N - 1); per dimension and bin, d_ji = sum of w^2 over
  the points whose coordinate j fell in bin i (the bin counts are kept too);
* refinement of each dimension: average d over N (d_i / N), smooth with
  neighbours ((d_0+d_1)/2, (d_{i-1}+d_i+d_{i+1})/3, (d_{N-2}+d_{N-1})/2),
  normalise to sum 1, compress r_i = ((r_i - 1) / ln r_i)^alpha with
  alpha = 1.5 (r_i = 0 stays 0, r_i = 1 gives 1), and place new edges so that
  each new bin holds an equal share of sum r, the old bins' content being
  spread uniformly inside each old bin;
* combination of iterations: inverse-variance weighted mean, its error, and
  chi^2 per degree of freedom.

The uniforms come from ``oracle.philox.vegas_uniforms``.
"""
from __future__ import annotations

import math

import numpy as np

from .philox import vegas_uniforms


def uniform_grid(ndim: int, nbins: int) -> np.ndarray:
    return np.tile(np.linspace(0.0, 1.0, nbins + 1), (ndim, 1))


def vegas_map(grid: np.ndarray, y: np.ndarray):
    """(x [d, N], jacobian [N], bins [d, N] int) for unit numbers y [d, N]."""
    d, nb1 = grid.shape
    nb = nb1 - 1
    y = np.asarray(y, dtype=np.float64)
    ynb = y * nb
    i = np.minimum(np.floor(ynb).astype(np.int64), nb - 1)
    rows = np.arange(d)[:, None]
    lo = grid[rows, i]
    width = grid[rows, i + 1] - lo
    x = lo + (ynb - i) * width
    jac = np.prod(nb * width, axis=0)
    return x, jac, i


def accumulate(w: np.ndarray, bins: np.ndarray, nbins: int):
    """Sums of one iteration: (sum w, sum w^2, d [dim, nb], counts [dim, nb])."""
    d = bins.shape[0]
    dsum = np.zeros((d, nbins))
    cnt = np.zeros((d, nbins), dtype=np.int64)
    w2 = w * w
    for j in range(d):
        dsum[j] = np.bincount(bins[j], weights=w2, minlength=nbins)
        cnt[j] = np.bincount(bins[j], minlength=nbins)
    return float(np.sum(w)), float(np.sum(w2)), dsum, cnt


def iteration_result(s1: float, s2: float, n: int):
    I = s1 / n
    var = (s2 / n - I * I) / (n - 1)
    return I, math.sqrt(max(var, 0.0))


def refine(grid: np.ndarray, dsum: np.ndarray, n: int, alpha: float = 1.5) -> np.ndarray:
    d, nb1 = grid.shape
    nb = nb1 - 1
    new = np.empty_like(grid)
    for j in range(d):
        avg = dsum[j] / n
        sm = np.empty(nb)
        sm[0] = (avg[0] + avg[1]) / 2.0
        sm[-1] = (avg[-2] + avg[-1]) / 2.0
        for i in range(1, nb - 1):
            sm[i] = (avg[i - 1] + avg[i] + avg[i + 1]) / 3.0
        tot = np.sum(sm)
        if tot <= 0.0:
            new[j] = grid[j]
            continue
        r = sm / tot
        comp = np.zeros(nb)
        for i in range(nb):
            if r[i] <= 0.0:
                comp[i] = 0.0
            elif r[i] == 1.0:
                comp[i] = 1.0
            else:
                comp[i] = ((r[i] - 1.0) / math.log(r[i])) ** alpha
        total = np.sum(comp)
        per_bin = total / nb
        # walk the old bins, placing an edge each time per_bin of content is reached
        edges = [0.0]
        acc = 0.0
        i_old = -1
        for k in range(1, nb):
            target = k * per_bin
            while acc < target:
                i_old += 1
                acc += comp[i_old]
            # the edge falls inside old bin i_old: content before it is acc - comp
            lo, hi = grid[j, i_old], grid[j, i_old + 1]
            frac = (target - (acc - comp[i_old])) / comp[i_old]
            edges.append(lo + frac * (hi - lo))
        edges.append(1.0)
        new[j] = np.array(edges)
    return new


def combine(results):
    """Inverse-variance weighted combination of [(I_k, sigma_k)]: (I, sigma, chi2/dof).

    Degenerate case: iterations with sigma_k = 0 are exact; if there are any,
    the result is their plain mean with zero error and chi^2/dof = 0.
    """
    I = np.array([r[0] for r in results])
    s = np.array([r[1] for r in results])
    exact = s == 0.0
    if np.any(exact):
        return float(np.mean(I[exact])), 0.0, 0.0
    wts = 1.0 / (s * s)
    mean = np.sum(wts * I) / np.sum(wts)
    err = 1.0 / math.sqrt(np.sum(wts))
    dof = len(results) - 1
    chi2 = float(np.sum(wts * (I - mean) ** 2) / dof) if dof > 0 else 0.0
    return float(mean), err, chi2


def run(f, ndim: int, n_events: int, n_iter: int, seed: int, nbins: int = 50,
        alpha: float = 1.5, subprocess: int = 0, grid=None, chunk: int = 1 << 16):
    """Full Vegas run of integrand f(x [d, N]) -> [N]. Returns dict of results."""
    grid = uniform_grid(ndim, nbins) if grid is None else np.array(grid, dtype=np.float64)
    per_iter = []
    hist = []
    for it in range(n_iter):
        s1 = s2 = 0.0
        dsum = np.zeros((ndim, nbins))
        cnt = np.zeros((ndim, nbins), dtype=np.int64)
        for start in range(0, n_events, chunk):
            m = min(chunk, n_events - start)
            y = vegas_uniforms(seed, it, subprocess, start, m, ndim)
            x, jac, bins = vegas_map(grid, y)
            w = f(x) * jac
            a, b, dd, cc = accumulate(w, bins, nbins)
            s1 += a
            s2 += b
            dsum += dd
            cnt += cc
        per_iter.append(iteration_result(s1, s2, n_events))
        hist.append((dsum, cnt, grid.copy()))
        if it != n_iter - 1:
            grid = refine(grid, dsum, n_events, alpha)
    mean, err, chi2 = combine(per_iter)
    return dict(iterations=per_iter, sigma=mean, error=err, chi2_dof=chi2, grid=grid, hist=hist)
