"""Per-event leading-order integrand (oracle).

Fig. 1 of the paper: the integrand is the parton luminosity L(x1, x2) times
the partonic cross section built from the matrix element and the RAMBO phase
space.  For a point x in the unit hypercube (no Vegas Jacobian here; Vegas
multiplies its own):

  hadronic:   (x1, x2, tau, J_x) = xmap(x_0, x_1, tau_min),  s-hat = tau S,
              tau_min = (sum of final masses)^2 / S
  lepton:     s-hat = S, J_x = 1, no densities
  momenta:    flat massless phase space from the remaining 3n-4 numbers,
              rescaled to the final-state masses (weight W)
  cuts:       every final gluon pT > pT_min, every final gluon pair
              Delta R = sqrt(Delta y^2 + Delta phi^2) > Delta R_min
              (Delta phi in (-pi, pi]); failing points get f = 0
  f(x)   =    J_x W f_1(x1, mu_F^2) f_2(x2, mu_F^2) |M|^2-bar / (2 s-hat)
              x 0.3893793721e9 pb GeV^2

Incoming partons are p_a = sqrt(s-hat)/2 (1,0,0,1), p_b = sqrt(s-hat)/2
(1,0,0,-1); outgoing momenta are those of the phase-space generator, in the
partonic centre-of-mass frame (the cuts are longitudinally boost invariant).
|M|^2-bar is averaged over initial spins and colours and carries 1/k! for k
identical final particles.
"""
from __future__ import annotations

import math

import numpy as np

import workloads as W
from . import phasespace as ps
from .feynman import Process, PARTICLES
from .pdf import PdfTable

MASSES_OF = {"t": "m_top"}


def oracle_process(wl: W.Workload, m_top=None, alpha_s=None) -> Process:
    mt = wl.m_top if m_top is None else m_top
    a_s = wl.alpha_s if alpha_s is None else alpha_s
    legs = [(l.particle, l.incoming) for l in wl.legs]
    return Process(legs, {"t": mt}, g_s=math.sqrt(4 * math.pi * a_s),
                   e=math.sqrt(4 * math.pi * wl.alpha))


def _pdf(name: str, q2_slope: float = 0.0) -> PdfTable:
    return PdfTable(W.pdf_table(name, q2_slope), W.PDF_X_MIN, W.PDF_X_MAX, W.PDF_Q2_MIN, W.PDF_Q2_MAX)


class Integrand:
    def __init__(self, wl: W.Workload, m_top=None, alpha_s=None, q2_slope: float = 0.0,
                 process: Process | None = None):
        self.wl = wl
        self.m_top = wl.m_top if m_top is None else m_top
        self.proc = process if process is not None else oracle_process(wl, m_top, alpha_s)
        if process is not None:
            self.proc.masses["t"] = self.m_top
        self.pdfs = tuple(_pdf(b, q2_slope) for b in wl.beams)
        self.final_masses = []
        for l in wl.legs:
            if not l.incoming:
                flav = PARTICLES[l.particle][1]
                self.final_masses.append(self.m_top if flav == "t" else 0.0)
        self.final_masses = np.array(self.final_masses)
        S = wl.sqrt_s ** 2
        self.S = S
        self.tau_min = (np.sum(self.final_masses) ** 2) / S if wl.beams else None
        self.gluon_finals = [i for i, l in enumerate(wl.legs) if not l.incoming and l.particle == "g"]

    # ------------------------------------------------------------------
    def use_channels(self, s0: float, t0: float):
        """Switch on the multichannel phase space of oracle/channels.py with
        regulators s0 (s-channel) and t0 (t-channel), GeV^2; returns the
        channels in their canonical order."""
        from . import channels as chmod
        self.channels = chmod.derive_channels(self.proc)
        self.s0, self.t0 = float(s0), float(t0)
        return self.channels

    def kinematics(self, x, final_masses=None, channel=None, masses=None):
        """Momenta [N, n, 4], s-hat, x1, x2, J_x and W for points x [ndim, N]
        (final-state masses as given, else the workload's).  With a channel
        index (after use_channels) the momenta come from that channel and W
        is a_i / g_i, the channel's share of the partition over its density."""
        from oracle.dual import as_f64
        x = as_f64(x)
        N = x.shape[1]
        fm = self.final_masses if final_masses is None else final_masses
        if self.wl.beams:
            msum = sum(fm[i] for i in range(len(fm)))
            tau_min = self.tau_min if final_masses is None else msum * msum / self.S
            x1, x2, tau, jx = ps.xmap(x[0], x[1], tau_min)
            s_hat = tau * self.S
            u = x[2:]
        else:
            x1 = x2 = np.ones(N)
            jx = np.ones(N)
            s_hat = np.full(N, self.S)
            u = x
        rs = np.sqrt(s_hat)
        n_out = self.wl.n_out
        if channel is not None:
            from . import channels as chmod
            mt = [self.m_top] if masses is None else masses
            k, inv_g, ok = chmod.generate(self.channels[channel], u, rs, fm, self.s0, self.t0, mt)
            pa = np.stack([rs / 2, 0 * rs, 0 * rs, rs / 2], axis=1)
            a = chmod.partition(self.channels, pa, k, self.s0, self.t0, mt)[:, channel]
            w = a * inv_g
        else:
            p0 = ps.massless_diet(u, rs)
            k, wfac, ok = ps.massive(p0, fm, rs)
            w = ps.massless_weight(n_out, s_hat) * wfac
        p = np.zeros((N, n_out + 2, 4), like=k)
        p[:, 0] = np.stack([rs / 2, 0 * rs, 0 * rs, rs / 2], axis=1)
        p[:, 1] = np.stack([rs / 2, 0 * rs, 0 * rs, -rs / 2], axis=1)
        p[:, 2:] = k
        return p, s_hat, x1, x2, jx, w, ok

    def cuts(self, p):
        N = p.shape[0]
        keep = np.ones(N, dtype=bool)
        wl = self.wl
        for i in self.gluon_finals:
            pt = np.hypot(p[:, i, 1], p[:, i, 2])
            keep &= pt > wl.pt_min_gluon
        if wl.dr_min_gluon > 0:
            # Delta R only where the pT cuts kept the point: there every
            # gluon has pT > 0, so its rapidity is finite (a gluon along the
            # beam has none)
            k = np.flatnonzero(keep)
            q = p[k]
            for a in range(len(self.gluon_finals)):
                for b in range(a + 1, len(self.gluon_finals)):
                    i, j = self.gluon_finals[a], self.gluon_finals[b]
                    yi = 0.5 * np.log((q[:, i, 0] + q[:, i, 3]) / (q[:, i, 0] - q[:, i, 3]))
                    yj = 0.5 * np.log((q[:, j, 0] + q[:, j, 3]) / (q[:, j, 0] - q[:, j, 3]))
                    dphi = np.arctan2(q[:, i, 2], q[:, i, 1]) - np.arctan2(q[:, j, 2], q[:, j, 1])
                    dphi = np.angle(np.exp(1j * dphi))
                    dr = np.sqrt((yi - yj) ** 2 + dphi ** 2)
                    keep[k] &= dr > wl.dr_min_gluon
        return keep

    def __call__(self, x, return_parts=False, channel=None):
        x = np.asarray(x, dtype=np.float64)
        N = x.shape[1]
        p, s_hat, x1, x2, jx, w, ok = self.kinematics(x, channel=channel)
        keep = ok & self.cuts(p)
        f = np.zeros(N)
        if np.any(keep):
            idx = np.nonzero(keep)[0]
            msq = self.proc.msq_avg(p[idx])
            lum = np.ones(len(idx))
            if self.wl.beams:
                lum = (self.pdfs[0].f(x1[idx], self.wl.mu_f2) * self.pdfs[1].f(x2[idx], self.wl.mu_f2))
            f[idx] = jx[idx] * w[idx] * lum * msq / (2.0 * s_hat[idx]) * W.GEV2_TO_PB
        if return_parts:
            cond = self.condition(p, s_hat, x1, x2)
            if channel is not None:
                cond = cond + self.channel_condition(s_hat)
            return f, dict(p=p, s_hat=s_hat, x1=x1, x2=x2, jx=jx, w=w, keep=keep,
                           pdf_condition=self._pdf_condition(x1, x2), condition=cond)
        return f

    def channel_condition(self, s_hat):
        """Bound on the condition number of a channel point's weight a_i / g_i:
        every propagator factor 1/(|x - M^2| + r)^2 of the partition and every
        t-channel density 1/(M^2 + t0 - t) moves by at most 2 eps s-hat / r
        when its invariant, formed from components up to sqrt(s-hat), moves by
        eps s-hat; summed over the largest channel's factors (numerator and
        denominator of the share, and the density)."""
        from . import channels as chmod
        n_fac = 0
        for ch in self.channels:
            n_prop = sum(1 for c in ch.spine for _ in chmod._clusters(c)) + ch.k - 1
            n_fac = max(n_fac, n_prop)
        return (3 * n_fac) * 2.0 * s_hat / min(self.s0, self.t0)

    # ------------------------------------------------------------------
    # derivatives by forward-mode dual numbers
    def gradient(self, x, channel=None):
        """(f [N], df/dx [ndim, N], df/dm_t [N]) at points x [ndim, N]: the
        integrand evaluated once in dual arithmetic with tangents along every
        coordinate of x and along the top mass (which enters the threshold
        tau_min, the phase-space rescaling, the spinors' momenta and the
        propagators; mu_F is held at its value).  Cut decisions are taken on
        values: the derivative is the pathwise one."""
        from oracle.dual import Dual
        x = np.asarray(x, dtype=np.float64)
        ndim, N = x.shape
        K = ndim + 1
        dx = np.zeros((ndim, N, K))
        for j in range(ndim):
            dx[j, :, j] = 1.0
        X = Dual(x, dx)
        mt = Dual(np.array(float(self.m_top)), np.eye(K)[ndim])
        fm = [mt if m > 0 else Dual(np.array(0.0), np.zeros(K)) for m in self.final_masses]
        saved = self.proc.masses
        self.proc.masses = {**saved, "t": mt}
        try:
            p, s_hat, x1, x2, jx, w, ok = self.kinematics(X, final_masses=fm, channel=channel, masses=[mt])
            pv = p.v if isinstance(p, Dual) else p
            keep = ok & self.cuts(pv)
            f = Dual(np.zeros(N), np.zeros((N, K)))
            idx = np.nonzero(keep)[0]
            if len(idx):
                msq = self.proc.msq_avg(p[idx])
                lum = 1.0
                if self.wl.beams:
                    lum = (self.pdfs[0].f(x1[idx], self.wl.mu_f2) * self.pdfs[1].f(x2[idx], self.wl.mu_f2))
                f[idx] = jx[idx] * w[idx] * lum * msq / (2.0 * s_hat[idx]) * W.GEV2_TO_PB
        finally:
            self.proc.masses = saved
        return f.v, np.moveaxis(f.d[:, :ndim], 1, 0), f.d[:, ndim]

    # ------------------------------------------------------------------
    # leading colour: the diagonal of the colour matrix in the string basis
    def leading_colour(self, x):
        x = np.asarray(x, dtype=np.float64)
        N = x.shape[1]
        p, s_hat, x1, x2, jx, w, ok = self.kinematics(x)
        keep = ok & self.cuts(p)
        f = np.zeros(N)
        idx = np.nonzero(keep)[0]
        if len(idx):
            msq = self.proc.msq_leading_colour(p[idx]) * self.proc.average_factor()
            lum = np.ones(len(idx))
            if self.wl.beams:
                lum = (self.pdfs[0].f(x1[idx], self.wl.mu_f2) * self.pdfs[1].f(x2[idx], self.wl.mu_f2))
            f[idx] = jx[idx] * w[idx] * lum * msq / (2.0 * s_hat[idx]) * W.GEV2_TO_PB
        return f

    # ------------------------------------------------------------------
    # helicity sampling: one helicity per point, uniform over a list of
    # non-vanishing helicities, |M_h|^2 scaled by the list's length (an
    # unbiased estimate of the helicity sum)
    def nonzero_helicities(self, n_points: int = 64, seed: int = 99):
        """Helicity assignments (in the oracle's order) whose |M|^2 does not
        vanish, judged on seeded random points passing the cuts; an
        assignment vanishes when it stays below 1e-12 of the helicity sum at
        every point (the explicit-matrix products leave rounding residues,
        ~1e-16 of the sum, where chirality makes an amplitude zero)."""
        rng = np.random.default_rng(seed)
        x = rng.random((self.wl.ndim, 4 * n_points))
        p, s_hat, x1, x2, jx, w, ok = self.kinematics(x)
        keep = ok & self.cuts(p)
        tot, per = self.proc.msq_summed(p[keep][:n_points], per_helicity=True)
        hels = self.proc.helicities()
        return [hels[h] for h in range(len(hels)) if np.any(np.abs(per[h]) > 1e-12 * tot)]

    def sampled(self, x, seed: int, helicities, pick=None, channel=None):
        """f with the helicity of point i drawn from the first unit number of
        Philox counter (i, 0, 0, 14), key (seed, 0) (or given by pick); with a
        channel index (after use_channels), through that phase-space channel."""
        from oracle.philox import philox4x64_10, to_unit
        x = np.asarray(x, dtype=np.float64)
        N = x.shape[1]
        nh = len(helicities)
        if pick is None:
            ctr = np.zeros((N, 4), dtype=np.uint64)
            ctr[:, 0] = np.arange(N, dtype=np.uint64)
            ctr[:, 3] = np.uint64(14)
            u = to_unit(philox4x64_10(ctr, np.array([seed, 0], dtype=np.uint64))[:, 0])
            pick = np.minimum((u * nh).astype(np.int64), nh - 1)
        p, s_hat, x1, x2, jx, w, ok = self.kinematics(x, channel=channel)
        keep = ok & self.cuts(p)
        f = np.zeros(N)
        idx = np.nonzero(keep)[0]
        if len(idx):
            order = {h: k for k, h in enumerate(self.proc.helicities())}
            _, per = self.proc.msq_summed(p[idx], per_helicity=True)
            rows = np.array([order[tuple(helicities[k])] for k in pick[idx]])
            msq = nh * per[rows, np.arange(len(idx))] * self.proc.average_factor()
            lum = np.ones(len(idx))
            if self.wl.beams:
                lum = (self.pdfs[0].f(x1[idx], self.wl.mu_f2) * self.pdfs[1].f(x2[idx], self.wl.mu_f2))
            f[idx] = jx[idx] * w[idx] * lum * msq / (2.0 * s_hat[idx]) * W.GEV2_TO_PB
        return f, pick

    def sampled_colour(self, x, seed: int, leading=False, pick=None):
        """f with the colour sum of every helicity replaced by the estimate
        from one colour string k per point: n_strings Re(conj(A_k) (G A)_k)
        (leading: n_strings G_kk |A_k|^2), k drawn uniformly from the first
        unit number of Philox counter (i, 0, 0, 12), key (seed, 0) (or given
        by pick); an unbiased estimate of f."""
        from oracle.philox import philox4x64_10, to_unit
        x = np.asarray(x, dtype=np.float64)
        N = x.shape[1]
        ns = self.proc.string_basis().shape[1]
        if pick is None:
            ctr = np.zeros((N, 4), dtype=np.uint64)
            ctr[:, 0] = np.arange(N, dtype=np.uint64)
            ctr[:, 3] = np.uint64(12)
            u = to_unit(philox4x64_10(ctr, np.array([seed, 0], dtype=np.uint64))[:, 0])
            pick = np.minimum((u * ns).astype(np.int64), ns - 1)
        p, s_hat, x1, x2, jx, w, ok = self.kinematics(x)
        keep = ok & self.cuts(p)
        f = np.zeros(N)
        idx = np.nonzero(keep)[0]
        if len(idx):
            if leading:
                rows = self.proc.leading_colour_weights(p[idx])[np.arange(len(idx)), pick[idx]]
            else:
                rows = self.proc.colour_row_sums(p[idx], pick[idx])
            msq = ns * rows * self.proc.average_factor()
            lum = np.ones(len(idx))
            if self.wl.beams:
                lum = (self.pdfs[0].f(x1[idx], self.wl.mu_f2) * self.pdfs[1].f(x2[idx], self.wl.mu_f2))
            f[idx] = jx[idx] * w[idx] * lum * msq / (2.0 * s_hat[idx]) * W.GEV2_TO_PB
        return f, pick

    @staticmethod
    def helicity_pairs(helicities, leg: int):
        """The helicity list grouped into pairs that differ only at `leg`
        (first member: helicity -1 there, second: +1; None where that
        assignment is not in the list), in the order of each pair's first row."""
        pairs, where = [], {}
        for h in helicities:
            key = tuple(v for l, v in enumerate(h) if l != leg)
            if key not in where:
                where[key] = len(pairs)
                pairs.append([None, None])
            pairs[where[key]][0 if h[leg] == -1 else 1] = tuple(h)
        return [tuple(q) for q in pairs]

    def sampled_pairs(self, x, seed: int, pairs, pick=None):
        """f with one helicity pair per point: pair pick[i] (drawn like the
        single helicity of `sampled`, from the first unit number of Philox
        counter (i, 0, 0, 14), over the pair list), its present members'
        |M_h|^2 summed and multiplied by the number of pairs (unbiased: the
        mean over the pairs is the full helicity sum)."""
        from oracle.philox import philox4x64_10, to_unit
        x = np.asarray(x, dtype=np.float64)
        N = x.shape[1]
        npair = len(pairs)
        if pick is None:
            ctr = np.zeros((N, 4), dtype=np.uint64)
            ctr[:, 0] = np.arange(N, dtype=np.uint64)
            ctr[:, 3] = np.uint64(14)
            u = to_unit(philox4x64_10(ctr, np.array([seed, 0], dtype=np.uint64))[:, 0])
            pick = np.minimum((u * npair).astype(np.int64), npair - 1)
        p, s_hat, x1, x2, jx, w, ok = self.kinematics(x)
        keep = ok & self.cuts(p)
        f = np.zeros(N)
        idx = np.nonzero(keep)[0]
        if len(idx):
            order = {h: k for k, h in enumerate(self.proc.helicities())}
            _, per = self.proc.msq_summed(p[idx], per_helicity=True)
            cols = np.arange(len(idx))
            msq = np.zeros(len(idx))
            for m in range(2):
                rows = [pairs[k][m] for k in pick[idx]]
                have = np.array([r is not None for r in rows])
                r_idx = np.array([order[r] if r is not None else 0 for r in rows])
                msq = msq + np.where(have, per[r_idx, cols], 0.0)
            msq = npair * msq * self.proc.average_factor()
            lum = np.ones(len(idx))
            if self.wl.beams:
                lum = (self.pdfs[0].f(x1[idx], self.wl.mu_f2) * self.pdfs[1].f(x2[idx], self.wl.mu_f2))
            f[idx] = jx[idx] * w[idx] * lum * msq / (2.0 * s_hat[idx]) * W.GEV2_TO_PB
        return f, pick

    # ------------------------------------------------------------------
    # condition numbers: how far two correct evaluations of f in different
    # operation orders can drift apart, in units of eps
    def _pdf_condition(self, x1, x2):
        if not self.wl.beams:
            return np.zeros(len(x1))
        with np.errstate(invalid="ignore", divide="ignore"):
            return self.pdfs[0].condition(x1, self.wl.mu_f2) + self.pdfs[1].condition(x2, self.wl.mu_f2)

    def condition(self, p, s_hat, x1, x2):
        """kappa_pdf + kappa_den + kappa_threshold per event:
        * PDF interpolation (cancellation and argument sensitivity);
        * propagator denominators q^2 - M^2 formed from summed components,
          (q0^2 + |q|^2 + M^2) / |q^2 - M^2|, maximised over every internal line;
        * production threshold: rs / (rs - sum of final masses), the relative
          precision of the final-state momenta near threshold."""
        N = p.shape[0]
        kp = self._pdf_condition(x1, x2)
        n = p.shape[1]
        sign = np.array([1.0 if inc else -1.0 for _, inc in self.proc.legs])
        masses = []
        for part, _ in self.proc.legs:
            kind, flav, _ = PARTICLES[part]
            masses.append(self.proc.masses.get(flav, 0.0) if kind == "F" else 0.0)
        kd = np.zeros(N)
        import itertools
        for r in range(2, n - 1):
            for S in itertools.combinations(range(n), r):
                q = np.sum(sign[list(S)][None, :, None] * p[:, list(S)], axis=1)
                big = q[:, 0] ** 2 + np.sum(q[:, 1:] ** 2, axis=1)
                q2 = q[:, 0] ** 2 - np.sum(q[:, 1:] ** 2, axis=1)
                for M in set([0.0] + [m for m in masses if m > 0]):
                    with np.errstate(divide="ignore", invalid="ignore"):
                        c = (big + M * M) / np.abs(q2 - M * M)
                    kd = np.maximum(kd, np.where(np.isfinite(c), c, 0.0))
        rs = np.sqrt(s_hat)
        ms = float(np.sum(self.final_masses))
        with np.errstate(divide="ignore", invalid="ignore"):
            kt = np.where(rs > ms, rs / (rs - ms), np.inf) if ms > 0 else np.ones(N)
        with np.errstate(invalid="ignore"):
            return kp + kd + kt
