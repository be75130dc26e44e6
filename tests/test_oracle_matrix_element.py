"""Pins of the oracle's brute-force |M|^2 (CPU only).

Closed forms: e+e- -> mu+mu- (photon only), gg -> tt~ and uu~ -> tt~ at
leading order (Combridge; Ellis, Stirling & Webber, Table 7.1/10.x).
Massless limit: the Parke-Taylor-type MHV partial amplitudes for one quark
line (L. Dixon, "Calculating scattering amplitudes efficiently", TASI 1995,
Sec. 4), combined with a brute-force SU(3) colour matrix, fix the colour- and
helicity-summed |M|^2 of q qbar g g exactly and of q qbar g g g exactly (every
non-zero helicity amplitude with five partons is MHV or anti-MHV).
Invariants: gauge invariance (eps -> k), Lorentz invariance, Bose symmetry.
"""
import itertools
import math

import numpy as np
import pytest

import workloads as W
from oracle import phasespace as ps
from oracle.feynman import Process, T_SU3, F_SU3
from oracle.integrand import Integrand

MD = np.array([1.0, -1.0, -1.0, -1.0])


def mdot(a, b):
    return np.einsum("...m,m,...m->...", a, MD, b)


def _points(wl, n, seed):
    I = Integrand(wl)
    x = W.uniform_points(wl.ndim, n, seed)
    p, s_hat, *_ = I.kinematics(x)
    return I, p, s_hat


# --------------------------------------------------------------- colour
def test_structure_constants_textbook_values():
    assert F_SU3[0, 1, 2] == pytest.approx(1.0, abs=1e-15)
    assert F_SU3[0, 3, 6] == pytest.approx(0.5, abs=1e-15)
    assert F_SU3[3, 4, 7] == pytest.approx(math.sqrt(3) / 2, abs=1e-15)
    assert np.allclose(F_SU3, -np.transpose(F_SU3, (1, 0, 2)), atol=1e-15)
    # Casimirs: t^a t^a = C_F 1, f^acd f^bcd = C_A delta
    assert np.allclose(np.einsum("aij,ajk->ik", T_SU3, T_SU3), 4 / 3 * np.eye(3), atol=1e-15)
    assert np.allclose(np.einsum("acd,bcd->ab", F_SU3, F_SU3), 3 * np.eye(8), atol=1e-14)


def trace_basis_colour_matrix(k):
    """C_st = sum_colours (t^s)_ij conj(t^t)_ij over orderings of k gluons."""
    perms = list(itertools.permutations(range(k)))
    vecs = []
    for perm in perms:
        arr = np.eye(3, dtype=complex)
        subs = []
        out = None
        # build (t^{a_perm0} ... t^{a_perm(k-1)})_{ij} as a tensor over (a_0..a_{k-1}, i, j)
        letters = "abcdefgh"
        expr = ",".join(f"{letters[g]}{'ijklmn'[pos]}{'ijklmn'[pos + 1]}" for pos, g in enumerate(perm))
        out_idx = "".join(letters[g] for g in range(k)) + "i" + "ijklmn"[k]
        vecs.append(np.einsum(expr + "->" + out_idx, *([T_SU3] * k)).ravel())
    V = np.stack(vecs, axis=1)
    return np.real(V.conj().T @ V), perms


def test_trace_basis_colour_matrices_known_values():
    C2, _ = trace_basis_colour_matrix(2)
    assert np.allclose(C2 * 3, [[16, -2], [-2, 16]], atol=1e-12)
    C3, _ = trace_basis_colour_matrix(3)
    assert set(np.unique(np.round(C3 * 9).astype(int))) == {64, -8, 10, 1}
    assert np.allclose(C3 * 9, np.round(C3 * 9), atol=1e-10)
    C4, _ = trace_basis_colour_matrix(4)
    vals = set(np.unique(np.round(C4 * 54).astype(int)))
    assert vals == {512, 80, 71, 62, 8, -1, -10, -28, -64}
    for C in (C2, C3, C4):
        assert np.min(np.linalg.eigvalsh(C)) > 0


# --------------------------------------------------------------- closed forms
def test_ee_mumu_closed_form():
    wl = W.EE_MUMU
    I, p, s = _points(wl, 300, 1)
    e2 = 4 * math.pi * wl.alpha
    t = mdot(p[:, 0] - p[:, 2], p[:, 0] - p[:, 2])
    u = mdot(p[:, 0] - p[:, 3], p[:, 0] - p[:, 3])
    ref = 2 * e2 ** 2 * (t * t + u * u) / s ** 2
    assert np.max(np.abs(I.proc.msq_avg(p) / ref - 1)) < 1e-13


def _tau_rho(p, s, m):
    t1 = 2 * mdot(p[:, 0], p[:, 2]) / s
    return t1, 1 - t1, 4 * m * m / s


def test_gg_ttx_closed_form():
    wl = W.GG_TTX
    I, p, s = _points(wl, 300, 2)
    t1, t2, rho = _tau_rho(p, s, wl.m_top)
    g4 = (4 * math.pi * wl.alpha_s) ** 2
    ref = g4 * (1 / (6 * t1 * t2) - 3 / 8) * (t1 ** 2 + t2 ** 2 + rho - rho ** 2 / (4 * t1 * t2))
    assert np.max(np.abs(I.proc.msq_avg(p) / ref - 1)) < 1e-12


def test_uux_ttx_closed_form():
    wl = W.UUX_TTX
    I, p, s = _points(wl, 300, 3)
    t1, t2, rho = _tau_rho(p, s, wl.m_top)
    g4 = (4 * math.pi * wl.alpha_s) ** 2
    ref = g4 * (4 / 9) * (t1 ** 2 + t2 ** 2 + rho / 2)
    assert np.max(np.abs(I.proc.msq_avg(p) / ref - 1)) < 1e-12


def test_gg_ttx_angular_integral_is_partonic_cross_section():
    # sigma-hat(gg -> QQ~) = pi a_s^2/(3 s) [(1 + rho + rho^2/16) ln((1+b)/(1-b)) - b (7/4 + 31 rho/16)]
    wl = W.GG_TTX
    proc = Integrand(wl).proc
    m, a_s = wl.m_top, wl.alpha_s
    for rs in (400.0, 900.0, 3000.0):
        s = rs * rs
        g, w = np.polynomial.legendre.leggauss(64)
        u = np.stack([0.5 * (g + 1), np.full_like(g, 0.3)])
        p0 = ps.massless_diet(u, np.full(64, rs))
        k, wfac, ok = ps.massive(p0, [m, m], rs)
        p = np.zeros((64, 4, 4))
        p[:, 0] = [rs / 2, 0, 0, rs / 2]
        p[:, 1] = [rs / 2, 0, 0, -rs / 2]
        p[:, 2:] = k
        msq = proc.msq_avg(p)
        W2 = ps.massless_weight(2, s) * wfac
        sig = np.sum(0.5 * w * W2 * msq) / (2 * s)
        rho = 4 * m * m / s
        b = math.sqrt(1 - rho)
        ref = math.pi * a_s ** 2 / (3 * s) * ((1 + rho + rho ** 2 / 16) * math.log((1 + b) / (1 - b))
                                              - b * (7 / 4 + 31 * rho / 16))
        assert sig == pytest.approx(ref, rel=1e-12)


# --------------------------------------------------------------- invariants
@pytest.mark.parametrize("name", ["gg_ttxg", "uux_ttxg", "gg_ttxgg"])
def test_gauge_invariance(name, oracle_processes):
    wl = W.WORKLOADS[name]
    proc = oracle_processes(name)
    I = Integrand(wl, process=proc)
    x = W.uniform_points(wl.ndim, 12, 5)
    p, *_ = I.kinematics(x)
    ref = proc.msq_summed(p)
    for leg, (part, inc) in enumerate(proc.legs):
        if part == "g":
            g = proc.msq_summed(p, gauge_leg=leg)
            assert np.max(np.abs(g / ref)) < 1e-12, (name, leg)


@pytest.mark.parametrize("name", ["gg_ttx", "gg_ttxg", "uux_ttxg", "gg_ttxgg"])
def test_lorentz_invariance(name, oracle_processes):
    wl = W.WORKLOADS[name]
    proc = oracle_processes(name)
    I = Integrand(wl, process=proc)
    x = W.uniform_points(wl.ndim, 10, 6)
    p, *_ = I.kinematics(x)
    ref = proc.msq_summed(p)
    rng = np.random.default_rng(7)
    for _ in range(2):
        beta = rng.uniform(-0.9, 0.9, 3) / math.sqrt(3)
        b2 = beta @ beta
        gam = 1 / math.sqrt(1 - b2)
        L = np.eye(4)
        L[0, 0] = gam
        L[0, 1:] = L[1:, 0] = gam * beta
        L[1:, 1:] += (gam - 1) * np.outer(beta, beta) / b2
        pb = np.einsum("ij,nkj->nki", L, p)
        got = proc.msq_summed(pb)
        assert np.max(np.abs(got / ref - 1)) < 1e-11


@pytest.mark.parametrize("name,pairs", [("gg_ttxg", [(0, 1)]), ("gg_ttxgg", [(0, 1), (4, 5)])])
def test_bose_symmetry(name, pairs, oracle_processes):
    wl = W.WORKLOADS[name]
    proc = oracle_processes(name)
    I = Integrand(wl, process=proc)
    x = W.uniform_points(wl.ndim, 10, 8)
    p, *_ = I.kinematics(x)
    ref = proc.msq_summed(p)
    for a, b in pairs:
        q = p.copy()
        q[:, [a, b]] = p[:, [b, a]]
        assert np.max(np.abs(proc.msq_summed(q) / ref - 1)) < 1e-12


def test_diagram_counts(oracle_processes):
    counts = {"ee_mumu": 1, "gg_ttx": 3, "uux_ttx": 1, "gg_ttxg": 16, "uux_ttxg": 5, "gg_ttxgg": 123}
    for name, c in counts.items():
        assert len(oracle_processes(name).diagrams) == c


# --------------------------------------------------------------- massless MHV
def _lam(k):
    """Spinors lambda, lambda-tilde of all-outgoing momenta (negative energy by
    analytic continuation with a factor i)."""
    sgn = np.sign(k[:, 0])
    kk = k * sgn[:, None]
    kp = kk[:, 0] + kk[:, 3]
    lam = np.stack([np.sqrt(kp), (kk[:, 1] + 1j * kk[:, 2]) / np.sqrt(kp)], axis=1).astype(complex)
    lt = np.conj(lam)
    neg = sgn < 0
    lam[neg] *= 1j
    lt[neg] *= 1j
    return lam, lt


def _ang(a, b):
    return a[:, 0] * b[:, 1] - a[:, 1] * b[:, 0]


def _mhv_total(k, qb, q, gluons, g):
    """Colour- and helicity-summed |M|^2 from MHV (and anti-MHV) partial amplitudes."""
    n = len(gluons) + 2
    lam = {}
    lt = {}
    for i in range(k.shape[1]):
        lam[i], lt[i] = _lam(k[:, i])
    C, perms = trace_basis_colour_matrix(len(gluons))
    pref = (2 * g * g) ** (n - 2)
    total = np.zeros(k.shape[0])
    brackets = [(lam, "mhv")] if n == 4 else [(lam, "mhv"), (lt, "anti")]
    for spin, _ in brackets:
        br = lambda a, b: _ang(spin[a], spin[b])
        for qneg in (True, False):
            for j in gluons:
                amps = []
                for perm in perms:
                    order = [qb] + [gluons[i] for i in perm] + [q]
                    den = np.ones(k.shape[0], dtype=complex)
                    for a, b in zip(order, order[1:] + order[:1]):
                        den = den * br(a, b)
                    num = br(qb, j) ** 3 * br(q, j) if qneg else br(qb, j) * br(q, j) ** 3
                    amps.append(1j * num / den)
                A = np.stack(amps)
                total += np.real(np.einsum("sn,st,tn->n", np.conj(A), C, A))
    return pref * total


@pytest.mark.parametrize("final", ["u u~", "u u~ g"])
def test_massless_mhv_formula(final):
    legs = [("g", True), ("g", True)] + [(p, False) for p in final.split()]
    g_s = 1.3
    proc = Process(legs, {}, g_s=g_s)
    n_out = len(legs) - 2
    rng = np.random.default_rng(31)
    N = 40
    rs = 1000.0
    pf = ps.massless_diet(rng.random((3 * n_out - 4, N)), rs)
    p = np.zeros((N, n_out + 2, 4))
    p[:, 0] = [rs / 2, 0, 0, rs / 2]
    p[:, 1] = [rs / 2, 0, 0, -rs / 2]
    p[:, 2:] = pf
    # random rotation so that no momentum lies on the z axis of the spinor formula
    A = np.linalg.qr(rng.normal(size=(3, 3)))[0]
    R = np.eye(4)
    R[1:, 1:] = A
    pr = np.einsum("ij,nkj->nki", R, p)
    ref = proc.msq_summed(p)
    k = pr.copy()
    k[:, :2] *= -1                      # all outgoing
    gluons = [i for i, (part, _) in enumerate(legs) if part == "g"]
    mhv = _mhv_total(k, qb=3, q=2, gluons=gluons, g=g_s)
    assert np.max(np.abs(mhv / ref - 1)) < 1e-11


def test_string_basis_norms_and_leading_colour(oracle_processes):
    # each basis element's squared norm is prod over its strings of
    # N C_F^m (m gluons on the string, C_F = 4/3); for uu~ -> tt~ the Fierz
    # identity gives the colour factor 1/2 B1 - 1/6 B2, so the leading-colour
    # sum (diagonal of the colour matrix in this basis) is 9/4 + 1/4 against
    # the full 2: a ratio of exactly 5/4 at every point
    import workloads as W
    from oracle.integrand import Integrand
    expect = {"gg_ttx": [16 / 3] * 2, "uux_ttx": [9.0] * 2, "uux_ttxg": [12.0] * 4, "gg_ttxg": [64 / 9] * 6,
              "gg_ttxgg": [256 / 27] * 24}
    for name, norms in expect.items():
        B = oracle_processes(name).string_basis()
        got = np.real(np.sum(np.conj(B) * B, axis=0))
        assert np.allclose(got, norms, rtol=1e-13), name
    I = Integrand(W.UUX_TTX, process=oracle_processes("uux_ttx"))
    x = W.uniform_points(4, 30, 8)
    full = I(x)
    lc = I.leading_colour(x)
    nz = full != 0
    assert np.allclose(lc[nz] / full[nz], 1.25, rtol=1e-12)


@pytest.mark.parametrize("name", ["gg_ttx", "uux_ttxg", "gg_ttxg"])
def test_colour_sampled_estimate_averages_to_the_colour_sum(name):
    # the mean over the strings of n_strings Re(conj(A_k) (G A)_k), from the
    # string-basis projection, equals the brute-force colour sum over
    # explicit colour assignments; likewise the leading-colour version
    import workloads as W
    from oracle.integrand import Integrand
    wl = W.WORKLOADS[name]
    I = Integrand(wl)
    x = W.uniform_points(wl.ndim, 25, 9)
    f, lc = I(x), I.leading_colour(x)
    ns = I.proc.string_basis().shape[1]
    tot = sum(I.sampled_colour(x, 1, pick=np.full(25, k))[0] for k in range(ns)) / ns
    totl = sum(I.sampled_colour(x, 1, leading=True, pick=np.full(25, k))[0] for k in range(ns)) / ns
    nz = f != 0
    assert np.allclose(tot[nz], f[nz], rtol=1e-13, atol=0)
    assert np.allclose(totl[nz], lc[nz], rtol=1e-13, atol=0)


def test_chunked_colour_matrix_equals_the_one_pass_sum():
    # the colour matrix summed over chunks of colour assignments (the first
    # gluon legs' colours held fixed in turn), as the oracle does for seven
    # legs, against the sum over the whole colour tensor
    import workloads as W
    from oracle.integrand import oracle_process
    full = oracle_process(W.GG_TTXG).colour_matrix()
    chunked = oracle_process(W.GG_TTXG)
    chunked.COLOUR_CHUNK = 4096                # forces chunks of one or two fixed gluon colours
    G = chunked.colour_matrix()
    assert np.allclose(G, full, rtol=0, atol=1e-12 * np.abs(full).max())


def test_seven_leg_oracle_counts_diagrams_and_is_gauge_invariant():
    # gg -> tt~ggg: 1240 Feynman diagrams; with a gluon's polarisation
    # replaced by its momentum every colour-dressed amplitude vanishes (here
    # on the colour assignments with the incoming gluons' colours fixed,
    # 4608 of the 294912: the whole colour tensor is never built)
    import workloads as W
    from oracle.integrand import oracle_process
    wl = W.GG_TTXGGG
    proc = oracle_process(wl)
    assert len(proc.diagrams) == 1240
    I = Integrand(wl, process=proc)
    x = W.uniform_points(wl.ndim, 8, 5)
    p, s_hat, x1, x2, jx, w, ok = I.kinematics(x)
    p = p[ok & I.cuts(p)][:2]
    Cc = proc._colour_columns({0: 3, 1: 5})
    hels = proc.helicities()
    for hi in (17, 100):
        A = Cc @ proc.amplitudes(p, hels[hi], {})
        for leg in (0, 1, 4, 5, 6):
            Ag = Cc @ proc.amplitudes(p, hels[hi], {}, gauge_leg=leg)
            assert np.abs(Ag).max() < 1e-12 * np.abs(A).max(), (hi, leg)
