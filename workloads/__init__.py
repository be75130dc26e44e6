"""Seeded synthetic inputs shared by the tests, the benchmark and the oracle.

This module holds input data only: physical parameters of the five
leading-order workloads, the synthetic parton-density tables that stand in
for the NNPDF grids the paper interpolates with PDFFlow (Sec. 2, Fig. 1), and
seeded uniform points in the unit hypercube.  It contains none of the
integrand's arithmetic (no phase space, no interpolation, no matrix element):
the CUDA library and the oracle each implement those independently.

Grids are stored row-major as ``table[iq][ix]`` (x fastest) with knots
uniform in ln x on [1e-6, 1] (100 knots) and uniform in ln Q^2 on
[1, 1e8] GeV^2 (50 knots).  The tabulated quantity is x f(x, Q^2).
"""
from __future__ import annotations

from dataclasses import dataclass, field
import math

import numpy as np

# --------------------------------------------------------------------------
# physical constants of the synthetic workloads
# --------------------------------------------------------------------------
GEV2_TO_PB = 0.3893793721e9      # 1 GeV^-2 in pb
SQRT_S_LHC = 13000.0             # GeV, hadronic centre-of-mass energy (Sec. 3)
SQRT_S_EE = 91.0                 # GeV, e+e- workload
M_TOP = 173.0                    # GeV
ALPHA_S = 0.118                  # fixed, no running
ALPHA_EM = 1.0 / 128.0

# PDF table geometry
PDF_NX = 100
PDF_NQ = 50
PDF_X_MIN = 1e-6
PDF_X_MAX = 1.0
PDF_Q2_MIN = 1.0
PDF_Q2_MAX = 1e8

# Normalisations chosen so that the gluon carries half of the proton momentum
# (int_0^1 x g dx = 0.5) and the valence-like up density counts two quarks
# (int_0^1 u dx = 2).  A = 0.5 / B(0.8, 6), B = 2 / B(0.5, 4) = 35/16.
PDF_A_GLUON = 0.5 * math.gamma(6.8) / (math.gamma(0.8) * math.gamma(6.0))
PDF_B_UP = 35.0 / 16.0


def x_knots() -> np.ndarray:
    return np.exp(np.linspace(math.log(PDF_X_MIN), math.log(PDF_X_MAX), PDF_NX))


def q2_knots() -> np.ndarray:
    return np.exp(np.linspace(math.log(PDF_Q2_MIN), math.log(PDF_Q2_MAX), PDF_NQ))


def xg_analytic(x):
    """Synthetic gluon: x g(x) = A x^-0.2 (1-x)^5, no Q^2 dependence."""
    x = np.asarray(x, dtype=np.float64)
    return PDF_A_GLUON * x ** (-0.2) * (1.0 - x) ** 5


def xu_analytic(x):
    """Synthetic valence-like up quark: x u(x) = B x^0.5 (1-x)^3."""
    x = np.asarray(x, dtype=np.float64)
    return PDF_B_UP * x ** 0.5 * (1.0 - x) ** 3


def pdf_table(name: str, q2_slope: float = 0.0) -> np.ndarray:
    """Tabulate x f on the (Q^2, x) knots, shape [PDF_NQ, PDF_NX], float64.

    ``q2_slope`` != 0 multiplies by (1 + q2_slope * ln(Q^2 / m_t^2)); it is a
    test-only variant that gives the table a Q^2 dependence so that the
    interpolation in ln Q^2 is exercised.
    """
    xs = x_knots()
    if name == "g":
        row = xg_analytic(xs)
    elif name in ("u", "ubar"):
        row = xu_analytic(xs)
    else:
        raise ValueError(f"unknown synthetic pdf {name!r}")
    row = row.copy()
    row[-1] = 0.0                     # (1-x)^k vanishes at x = 1 exactly
    qs = q2_knots()
    fac = 1.0 + q2_slope * np.log(qs / M_TOP ** 2)
    return np.ascontiguousarray(fac[:, None] * row[None, :])


# --------------------------------------------------------------------------
# workload (process) parameter sets
# --------------------------------------------------------------------------
@dataclass(frozen=True)
class Leg:
    particle: str   # 'g', 'a' (photon), 'u', 'u~', 't', 't~', 'e-', 'e+', 'mu-', 'mu+'
    incoming: bool


@dataclass(frozen=True)
class Workload:
    name: str
    legs: tuple            # tuple[Leg, ...]; incoming legs first
    sqrt_s: float          # collider energy in GeV
    beams: tuple           # ('g','g'), ('u','ubar') or () for a lepton collider
    mu_f2: float           # factorisation scale squared
    m_top: float = M_TOP
    alpha_s: float = ALPHA_S
    alpha: float = ALPHA_EM
    pt_min_gluon: float = 0.0      # pT cut on every final-state gluon
    dr_min_gluon: float = 0.0      # Delta R cut between final-state gluon pairs
    n_events: int = 0              # events per Vegas iteration
    n_iter: int = 0
    n_bins: int = 50
    alpha_vegas: float = 1.5
    extra: dict = field(default_factory=dict, hash=False, compare=False)

    @property
    def n_out(self) -> int:
        return sum(1 for l in self.legs if not l.incoming)

    @property
    def ndim(self) -> int:
        """Vegas dimensions: 3 n_out - 4 phase-space numbers, + 2 for x1, x2."""
        return 3 * self.n_out - 4 + (2 if self.beams else 0)


def _legs(spec: str) -> tuple:
    ins, outs = spec.split("->")
    return tuple([Leg(p, True) for p in ins.split()] + [Leg(p, False) for p in outs.split()])


EE_MUMU = Workload("ee_mumu", _legs("e- e+ -> mu- mu+"), SQRT_S_EE, (), SQRT_S_EE ** 2,
                   n_events=100_000, n_iter=5)
GG_TTX = Workload("gg_ttx", _legs("g g -> t t~"), SQRT_S_LHC, ("g", "g"), M_TOP ** 2,
                  n_events=1_000_000, n_iter=10)
UUX_TTX = Workload("uux_ttx", _legs("u u~ -> t t~"), SQRT_S_LHC, ("u", "ubar"), M_TOP ** 2,
                   n_events=5_000_000, n_iter=10)
GG_TTXG = Workload("gg_ttxg", _legs("g g -> t t~ g"), SQRT_S_LHC, ("g", "g"), M_TOP ** 2,
                   pt_min_gluon=20.0, n_events=10_000_000, n_iter=10)
UUX_TTXG = Workload("uux_ttxg", _legs("u u~ -> t t~ g"), SQRT_S_LHC, ("u", "ubar"), M_TOP ** 2,
                    pt_min_gluon=20.0, n_events=3_000_000, n_iter=10)
GG_TTXGG = Workload("gg_ttxgg", _legs("g g -> t t~ g g"), SQRT_S_LHC, ("g", "g"), M_TOP ** 2,
                    pt_min_gluon=20.0, dr_min_gluon=0.4, n_events=40_000_000, n_iter=10)

# the heavier workload of the paper's Sec. 3.2 (its pp -> tt~ggg with 100k
# events): the gg channel, 1240 diagrams, 120 colour flows
GG_TTXGGG = Workload("gg_ttxggg", _legs("g g -> t t~ g g g"), SQRT_S_LHC, ("g", "g"), M_TOP ** 2,
                     pt_min_gluon=20.0, dr_min_gluon=0.4, n_events=100_000, n_iter=10)

WORKLOADS = {w.name: w for w in (EE_MUMU, GG_TTX, UUX_TTX, GG_TTXG, UUX_TTXG, GG_TTXGG, GG_TTXGGG)}

# the mixed batch: one persistent launch over five subprocesses
MIXED_BATCH = (("gg_ttx", 20_000_000), ("uux_ttx", 5_000_000), ("gg_ttxg", 10_000_000),
               ("uux_ttxg", 3_000_000), ("gg_ttxgg", 2_000_000))


# --------------------------------------------------------------------------
# seeded points
# --------------------------------------------------------------------------
def uniform_points(ndim: int, n: int, seed: int) -> np.ndarray:
    """Seeded points in the open unit hypercube, structure-of-arrays [ndim, n]."""
    rng = np.random.Generator(np.random.PCG64(seed))
    u = rng.random((ndim, n))
    return np.ascontiguousarray(np.clip(u, 1e-15, 1.0 - 1e-15))


def edge_points(ndim: int) -> np.ndarray:
    """Corner-ish points (every coordinate near 0, 1/2 or 1), SoA [ndim, n]."""
    vals = np.array([1e-12, 0.5, 1.0 - 1e-12])
    rng = np.random.Generator(np.random.PCG64(12345))
    n = 64
    pts = vals[rng.integers(0, 3, size=(ndim, n))]
    return np.ascontiguousarray(pts)
