"""Log-bicubic interpolation of a parton-density table (oracle).

The paper evaluates PDFs with PDFFlow on the GPU (Sec. 1, Sec. 2.2 and the
"PDF" arrow of Fig. 1) but prints no interpolation formula; this oracle takes
the LHAPDF-style reading used by PDFFlow:

* knots uniform in a = ln x (nx knots on [x_min, x_max]) and in b = ln Q^2
  (nq knots on [q2_min, q2_max]); the table holds v[j][i] = x f(x_i, Q^2_j);
* knot derivatives by central differences, one-sided at the two end knots;
* a cubic Hermite polynomial in a along each Q^2 row j-1 .. j+2 around the
  query, then a cubic Hermite polynomial in b through those row values, with
  b-derivatives again from central (one-sided at the ends) differences;
* the density returned is f = (x f) / x.

Queries outside the table use the edge interval's cubic (index clamped).

Pinned in tests: exact at knots; exact for data that is biquadratic in
(ln x, ln Q^2) on interior intervals and bilinear everywhere; small error
against the analytic synthetic density between knots.
"""
from __future__ import annotations

import math

import numpy as np

from oracle.dual import as_f64


def _hermite(t, h, v0, v1, d0, d1):
    """Cubic Hermite on one interval: values v0, v1 and slopes d0, d1 (per unit
    of the abscissa), interval length h, local coordinate t in [0, 1]."""
    t2 = t * t
    t3 = t2 * t
    h00 = 2.0 * t3 - 3.0 * t2 + 1.0
    h10 = t3 - 2.0 * t2 + t
    h01 = -2.0 * t3 + 3.0 * t2
    h11 = t3 - t2
    return h00 * v0 + h10 * h * d0 + h01 * v1 + h11 * h * d1


def _knot_slope(vals, knots, k):
    """Central difference at knot k; one-sided at the ends (vals indexable)."""
    n = len(knots)
    if k == 0:
        return (vals[1] - vals[0]) / (knots[1] - knots[0])
    if k == n - 1:
        return (vals[n - 1] - vals[n - 2]) / (knots[n - 1] - knots[n - 2])
    return (vals[k + 1] - vals[k - 1]) / (knots[k + 1] - knots[k - 1])


class PdfTable:
    def __init__(self, table, x_min, x_max, q2_min, q2_max):
        self.v = np.asarray(table, dtype=np.float64)          # [nq, nx]
        self.nq, self.nx = self.v.shape
        self.a = np.array([math.log(x_min) + i * (math.log(x_max) - math.log(x_min)) / (self.nx - 1)
                           for i in range(self.nx)])
        self.b = np.array([math.log(q2_min) + j * (math.log(q2_max) - math.log(q2_min)) / (self.nq - 1)
                           for j in range(self.nq)])

    def _interval(self, knots, c):
        i = np.searchsorted(knots, c, side="right") - 1
        return np.clip(i, 0, len(knots) - 2)

    def _row_interp(self, j, i, a):
        """Hermite in ln x along table row j (vectorised over events)."""
        row = self.v[j]                       # [N, nx] via fancy indexing below
        n = self.nx
        idx = np.arange(len(a))
        v0 = row[idx, i]
        v1 = row[idx, i + 1]
        # slopes at knots i and i+1, central differences, one-sided at the ends
        def slope(k):
            lo = np.maximum(k - 1, 0)
            hi = np.minimum(k + 1, n - 1)
            return (row[idx, hi] - row[idx, lo]) / (self.a[hi] - self.a[lo])
        d0 = slope(i)
        d1 = slope(i + 1)
        h = self.a[i + 1] - self.a[i]
        t = (a - self.a[i]) / h
        return _hermite(t, h, v0, v1, d0, d1)

    def xfx(self, x, q2):
        """x f(x, Q^2), vectorised."""
        x = np.atleast_1d(as_f64(x))
        q2 = np.broadcast_to(np.asarray(q2, dtype=np.float64), x.shape)
        a = np.log(x)
        b = np.log(q2)
        i = self._interval(self.a, a)
        j = self._interval(self.b, b)
        # row values g_k at Q^2 knots k = j-1 .. j+2 (clamped to the table)
        g = {}
        for off in (-1, 0, 1, 2):
            k = np.clip(j + off, 0, self.nq - 1)
            g[off] = self._row_interp(k, i, a)
        # b-slopes at knots j and j+1
        def bslope(off):
            k = j + off
            lo_off = np.where(k - 1 < 0, off, off - 1)
            hi_off = np.where(k + 1 > self.nq - 1, off, off + 1)
            lo_val = np.choose(lo_off + 1, [g[-1], g[0], g[1], g[2]])
            hi_val = np.choose(hi_off + 1, [g[-1], g[0], g[1], g[2]])
            return (hi_val - lo_val) / (self.b[j + hi_off] - self.b[j + lo_off])
        e0 = bslope(0)
        e1 = bslope(1)
        h = self.b[j + 1] - self.b[j]
        t = (b - self.b[j]) / h
        return _hermite(t, h, g[0], g[1], e0, e1)

    def condition(self, x, q2):
        """Condition number of the interpolated value: the same interpolation
        with every coefficient and table entry replaced by its absolute value
        (slopes by (|v_hi| + |v_lo|)/Delta), divided by |x f|, plus the relative
        sensitivity to a rounding-sized change of ln x.  Two evaluations of
        the same definition in different operation orders agree to a small
        multiple of eps times this."""
        x = np.atleast_1d(as_f64(x))
        q2 = np.broadcast_to(np.asarray(q2, dtype=np.float64), x.shape)
        a, b = np.log(x), np.log(q2)
        i = self._interval(self.a, a)
        j = self._interval(self.b, b)
        idx = np.arange(len(a))

        def absherm(t, h, v0, v1, d0, d1):
            t2, t3 = t * t, t * t * t
            return (np.abs(2 * t3 - 3 * t2 + 1) * v0 + np.abs(t3 - 2 * t2 + t) * h * d0
                    + np.abs(-2 * t3 + 3 * t2) * v1 + np.abs(t3 - t2) * h * d1)

        def absrow(k):
            row = np.abs(self.v[k])
            n = self.nx
            def sl(kk):
                lo = np.maximum(kk - 1, 0)
                hi = np.minimum(kk + 1, n - 1)
                return (row[idx, hi] + row[idx, lo]) / (self.a[hi] - self.a[lo])
            h = self.a[i + 1] - self.a[i]
            return absherm((a - self.a[i]) / h, h, row[idx, i], row[idx, i + 1], sl(i), sl(i + 1))

        g = {off: absrow(np.clip(j + off, 0, self.nq - 1)) for off in (-1, 0, 1, 2)}

        def bsl(off):
            lo = np.clip(j + off - 1, 0, self.nq - 1)
            hi = np.clip(j + off + 1, 0, self.nq - 1)
            lo_v = np.choose(np.clip(lo - j + 1, 0, 3), [g[-1], g[0], g[1], g[2]])
            hi_v = np.choose(np.clip(hi - j + 1, 0, 3), [g[-1], g[0], g[1], g[2]])
            return (hi_v + lo_v) / (self.b[hi] - self.b[lo])
        h = self.b[j + 1] - self.b[j]
        tot = absherm((b - self.b[j]) / h, h, g[0], g[1], bsl(0), bsl(1))
        val = np.abs(self.xfx(x, q2))
        # sensitivity to the argument: |d(xf)/d ln x| for a perturbation of
        # ln x of relative size eps (absolute eps max(|ln x|, 1))
        d = 1e-6
        slope = np.abs(self.xfx(x * np.exp(d), q2) - self.xfx(x * np.exp(-d), q2)) / (2 * d)
        return tot / val + slope * np.maximum(np.abs(a), 1.0) / val

    def f(self, x, q2):
        """Number density f(x, Q^2) = (x f) / x."""
        x = np.atleast_1d(as_f64(x))
        return self.xfx(x, q2) / x


def xfx_scalar(table: PdfTable, x: float, q2: float) -> float:
    """Same definition evaluated with plain scalar loops (cross-check of the
    vectorised index bookkeeping above on single points)."""
    a, b = math.log(x), math.log(q2)
    i = min(max(int(np.searchsorted(table.a, a, side="right")) - 1, 0), table.nx - 2)
    j = min(max(int(np.searchsorted(table.b, b, side="right")) - 1, 0), table.nq - 2)
    rows = {}
    for k in range(max(j - 1, 0), min(j + 2, table.nq - 1) + 1):
        r = table.v[k]
        d0 = _knot_slope(r, table.a, i)
        d1 = _knot_slope(r, table.a, i + 1)
        h = table.a[i + 1] - table.a[i]
        rows[k] = _hermite((a - table.a[i]) / h, h, r[i], r[i + 1], d0, d1)

    def bslope(k):
        lo = k - 1 if k - 1 >= 0 else k
        hi = k + 1 if k + 1 <= table.nq - 1 else k
        return (rows[hi] - rows[lo]) / (table.b[hi] - table.b[lo])

    h = table.b[j + 1] - table.b[j]
    return _hermite((b - table.b[j]) / h, h, rows[j], rows[j + 1], bslope(j), bslope(j + 1))
