"""Tree-level |M|^2 by brute force (oracle).

The paper's ``smatrix`` (Sec. 2.3) loops over helicities and sums diagram
contributions built from HELAS/ALOHA wavefunctions and vertices.  The plain
definition of the quantity it returns is

    sum over colours and helicities of | sum over Feynman diagrams |^2 ,

and that is what this module writes out, with nothing reorganised:

* every tree diagram of the process is enumerated from the QCD vertices
  (q-qbar-g, ggg, gggg) or the QED vertex (l-lbar-photon);
* each diagram's kinematic factor is the product of textbook Feynman rules
  (Peskin & Schroeder conventions, covariant derivative d - i g A^a t^a):
    quark-gluon vertex        i g_s gamma^mu t^a
    three-gluon vertex        g_s f^abc [g^mn (k1-k2)^r + g^nr (k2-k3)^m
                                          + g^rm (k3-k1)^n]   (all k incoming)
    four-gluon vertex         -i g_s^2 [f^abe f^cde (g^mr g^ns - g^ms g^nr)
                                        + f^ace f^bde (g^mn g^rs - g^ms g^nr)
                                        + f^ade f^bce (g^mn g^rs - g^mr g^ns)]
    lepton-photon vertex      i e gamma^mu           (charge -1)
    gluon / photon propagator -i g_mn / k^2          (Feynman gauge)
    fermion propagator        i (q-slash + m) / (q^2 - m^2)
  evaluated with explicit 4x4 Dirac matrices (chiral representation);
* each diagram's colour factor is an explicit tensor over all external colour
  indices, contracted from Gell-Mann t^a = lambda^a / 2 and
  f^abc = -2i Tr([t^a, t^b] t^c); a four-gluon vertex splits a diagram into its
  three colour structures ("terms");
* sum_colours |sum_t c_t a_t|^2 = a^H G a with G = C^H C summed over every
  external colour assignment.

External states are helicity eigenstates: spinors u, v from two-component
helicity eigenvectors chi_lambda (HELAS conventions, KEK-91-11), transverse
polarisation vectors eps(k, +-1) = (-+ e1 - i e2)/sqrt 2 for incoming and their
conjugates for outgoing vector bosons.  Helicity-summed results do not depend
on these phase choices.

Pinned in tests by closed forms (e+e- -> mu+mu-, gg -> tt~, uu~ -> tt~),
the massless Parke-Taylor-type MHV formula (q qbar g g and q qbar g g g),
gauge invariance, Lorentz invariance, Bose symmetry and diagram counts.
"""
from __future__ import annotations

import itertools
import os
import math
from functools import lru_cache

import numpy as np

# ----------------------------------------------------------------------------
# SU(3)
# ----------------------------------------------------------------------------

def gell_mann() -> np.ndarray:
    l = np.zeros((8, 3, 3), dtype=np.complex128)
    l[0][0, 1] = l[0][1, 0] = 1
    l[1][0, 1] = -1j; l[1][1, 0] = 1j
    l[2][0, 0] = 1; l[2][1, 1] = -1
    l[3][0, 2] = l[3][2, 0] = 1
    l[4][0, 2] = -1j; l[4][2, 0] = 1j
    l[5][1, 2] = l[5][2, 1] = 1
    l[6][1, 2] = -1j; l[6][2, 1] = 1j
    l[7][0, 0] = l[7][1, 1] = 1 / math.sqrt(3); l[7][2, 2] = -2 / math.sqrt(3)
    return l


T_SU3 = gell_mann() / 2.0
F_SU3 = np.real(-2j * (np.einsum("aij,bjk,cki->abc", T_SU3, T_SU3, T_SU3)
                       - np.einsum("bij,ajk,cki->abc", T_SU3, T_SU3, T_SU3)))
# the three colour structures of the four-gluon vertex, legs (a, b, c, d)
F4_SU3 = np.stack([
    np.einsum("abe,cde->abcd", F_SU3, F_SU3),
    np.einsum("ace,bde->abcd", F_SU3, F_SU3),
    np.einsum("ade,bce->abcd", F_SU3, F_SU3),
])

# ----------------------------------------------------------------------------
# Dirac algebra, chiral representation, metric (+,-,-,-)
# ----------------------------------------------------------------------------
_I2 = np.eye(2, dtype=np.complex128)
_Z2 = np.zeros((2, 2), dtype=np.complex128)
SIGMA = np.array([[[0, 1], [1, 0]], [[0, -1j], [1j, 0]], [[1, 0], [0, -1]]], dtype=np.complex128)
GAMMA = np.stack([np.block([[_Z2, _I2], [_I2, _Z2]])]
                 + [np.block([[_Z2, SIGMA[k]], [-SIGMA[k], _Z2]]) for k in range(3)])
METRIC = np.array([1.0, -1.0, -1.0, -1.0])


def mdot(a, b):
    """Minkowski product without complex conjugation, [..., 4] x [..., 4]."""
    return a[..., 0] * b[..., 0] - a[..., 1] * b[..., 1] - a[..., 2] * b[..., 2] - a[..., 3] * b[..., 3]


def slash(a):
    """gamma^mu a_mu for contravariant a [N, 4] -> [N, 4, 4]."""
    return np.einsum("m,mij,nm->nij", METRIC, GAMMA, a)


# ----------------------------------------------------------------------------
# external wavefunctions
# ----------------------------------------------------------------------------

def _chi(p, lam):
    """Two-component helicity eigenvectors of sigma.p-hat, [N, 2]."""
    px, py, pz = p[:, 1], p[:, 2], p[:, 3]
    P = np.sqrt(px * px + py * py + pz * pz)
    pt2 = px * px + py * py
    # P + pz without cancellation when pz < 0
    ppz = np.where(pz >= 0, P + pz, pt2 / np.where(P - pz > 0, P - pz, 1.0))
    good = ppz > 0
    den = np.sqrt(np.where(good, 2.0 * P * ppz, 1.0))
    out = np.zeros((len(px), 2), dtype=np.complex128, like=px)
    if lam == 1:
        out[:, 0] = np.where(good, ppz / den, 0.0)
        out[:, 1] = np.where(good, (px + 1j * py) / den, 1.0)
    else:
        out[:, 0] = np.where(good, (-px + 1j * py) / den, -1.0)
        out[:, 1] = np.where(good, ppz / den, 0.0)
    at_rest = P == 0
    if np.any(at_rest):
        out[at_rest] = [1.0, 0.0] if lam == 1 else [0.0, 1.0]
    return out, P


def spinor_u(p, m, lam):
    chi, P = _chi(p, lam)
    E = p[:, 0]
    a = np.sqrt(np.maximum(E - lam * P, 0.0))
    b = np.sqrt(np.maximum(E + lam * P, 0.0))
    return np.concatenate([a[:, None] * chi, b[:, None] * chi], axis=1)


def spinor_v(p, m, lam):
    chi, P = _chi(p, -lam)
    E = p[:, 0]
    c = -lam * np.sqrt(np.maximum(E + lam * P, 0.0))
    d = lam * np.sqrt(np.maximum(E - lam * P, 0.0))
    return np.concatenate([c[:, None] * chi, d[:, None] * chi], axis=1)


def bar(psi):
    """Dirac adjoint psi^dagger gamma^0 as a row [N, 4]."""
    return np.einsum("ni,ij->nj", np.conj(psi), GAMMA[0])


def polarisation(k, lam):
    """eps^mu(k, lam) for a massless vector boson, lam = +-1, [N, 4] complex."""
    kx, ky, kz = k[:, 1], k[:, 2], k[:, 3]
    K = np.sqrt(kx * kx + ky * ky + kz * kz)
    kt = np.sqrt(kx * kx + ky * ky)
    has_t = kt > 0
    sth = np.where(has_t, kt / np.where(K > 0, K, 1.0), 0.0)
    cth = np.where(has_t, kz / np.where(K > 0, K, 1.0), np.where(kz >= 0, 1.0, -1.0))
    cph = np.where(has_t, kx / np.where(has_t, kt, 1.0), 1.0)
    sph = np.where(has_t, ky / np.where(has_t, kt, 1.0), 0.0)
    zero = np.zeros_like(kx)
    e1 = np.stack([zero, cth * cph, cth * sph, -sth], axis=1)
    e2 = np.stack([zero, -sph, cph, zero], axis=1)
    return (-lam * e1 - 1j * e2) / math.sqrt(2.0)


# ----------------------------------------------------------------------------
# particles and lines
# ----------------------------------------------------------------------------
# name -> (kind, flavour, is_antiparticle)
PARTICLES = {
    "g": ("V", "g", False), "a": ("V", "a", False),
    "u": ("F", "u", False), "u~": ("F", "u", True),
    "t": ("F", "t", False), "t~": ("F", "t", True),
    "e-": ("F", "e", False), "e+": ("F", "e", True),
    "mu-": ("F", "mu", False), "mu+": ("F", "mu", True),
}
BOSON_OF = {"u": "g", "t": "g", "e": "a", "mu": "a"}
COLOUR_DIM = {"g": 8, "a": 1, "u": 3, "t": 3, "e": 1, "mu": 1}


def ext_line(particle: str, incoming: bool):
    kind, flav, anti = PARTICLES[particle]
    if kind == "V":
        return ("V", flav)
    # column spinor (u of an incoming particle, v of an outgoing antiparticle)
    column = (incoming and not anti) or (not incoming and anti)
    return ("F", flav, "in" if column else "out")


def _partner(line):
    if line[0] == "V":
        return line
    return ("F", line[1], "out" if line[2] == "in" else "in")


def _splits2(S):
    """Ordered splits of frozenset S into two non-empty parts."""
    items = sorted(S)
    out = []
    for r in range(1, len(items)):
        for A in itertools.combinations(items, r):
            A = frozenset(A)
            out.append((A, S - A))
    return out


def _unordered2(S):
    items = sorted(S)
    first = items[0]
    rest = items[1:]
    out = []
    for r in range(0, len(rest)):
        for extra in itertools.combinations(rest, r):
            A = frozenset((first,) + extra)
            B = S - A
            if B:
                out.append((A, B))
    return out


def _unordered3(S):
    out = []
    for A, BC in _unordered2(S):
        if len(BC) < 2:
            continue
        for B, C in _unordered2(BC):
            out.append((A, B, C))
    return out


def _colour_gram_part(args):
    """Sum over the given colour chunks of C^dagger C (see
    Process.colour_matrix)."""
    proc, chunks = args
    G = np.zeros((len(proc.terms), len(proc.terms)), dtype=np.complex128)
    for fixed in chunks:
        Cc = proc._colour_columns(fixed)
        G += Cc.conj().T @ Cc
    return G


class Process:
    """All tree diagrams of a 2 -> n process and the brute-force |M|^2."""

    def __init__(self, legs, masses: dict, g_s: float = 0.0, e: float = 0.0):
        # legs: sequence of (particle name, incoming flag); incoming first
        self.legs = [(p, bool(inc)) for p, inc in legs]
        self.n = len(self.legs)
        self.masses = dict(masses)
        self.g_s = g_s
        self.e = e
        self.lines = [ext_line(p, inc) for p, inc in self.legs]
        self.flavours = {PARTICLES[p][1] for p, _ in self.legs if PARTICLES[p][0] == "F"}
        self._memo = {}
        root = self.n - 1
        rest = frozenset(range(self.n - 1))
        need = _partner(self.lines[root])
        self.diagrams = [t for t in self._trees(rest, need) if t[0] == "N"]
        self.terms = []
        for d in self.diagrams:
            self.terms.extend(self._expand(d))
        self._G = None

    # ---------------------------------------------------------------- topology
    def _trees(self, S, line):
        key = (S, line)
        if key in self._memo:
            return self._memo[key]
        out = []
        if len(S) == 1:
            (leg,) = S
            if self.lines[leg] == line:
                out.append(("L", leg))
            self._memo[key] = out
            return out
        if line[0] == "F":
            flav, direction = line[1], line[2]
            boson = BOSON_OF[flav]
            for A, B in _splits2(S):
                for tf in self._trees(A, line):
                    for tv in self._trees(B, ("V", boson)):
                        out.append(("N", "fin" if direction == "in" else "fout", line, (tf, tv), 0))
        else:
            b = line[1]
            for flav in sorted(self.flavours):
                if BOSON_OF[flav] != b:
                    continue
                for A, B in _splits2(S):
                    for tc in self._trees(A, ("F", flav, "in")):
                        for tr in self._trees(B, ("F", flav, "out")):
                            out.append(("N", "vec", line, (tc, tr), 0))
            if b == "g":
                for A, B in _unordered2(S):
                    for ta in self._trees(A, ("V", "g")):
                        for tb in self._trees(B, ("V", "g")):
                            out.append(("N", "vvv", line, (ta, tb), 0))
                if len(S) >= 3:
                    for A, B, C in _unordered3(S):
                        for ta in self._trees(A, ("V", "g")):
                            for tb in self._trees(B, ("V", "g")):
                                for tc in self._trees(C, ("V", "g")):
                                    out.append(("N", "vvvv", line, (ta, tb, tc), 0))
        self._memo[key] = out
        return out

    def _expand(self, tree):
        """Split every four-gluon vertex into its three colour structures."""
        if tree[0] == "L":
            return [tree]
        _, kind, line, children, _ = tree
        child_opts = [self._expand(c) for c in children]
        out = []
        variants = (1, 2, 3) if kind == "vvvv" else (0,)
        for combo in itertools.product(*child_opts):
            for v in variants:
                out.append(("N", kind, line, tuple(combo), v))
        return out

    @staticmethod
    @lru_cache(maxsize=None)
    def legs_of(tree):
        if tree[0] == "L":
            return (tree[1],)
        return tuple(sorted(sum((Process.legs_of(c) for c in tree[3]), ())))

    # ---------------------------------------------------------------- colour
    def _colour_dim_leg(self, leg):
        p, _ = self.legs[leg]
        return COLOUR_DIM[PARTICLES[p][1]]

    def _generators(self, boson):
        if boson == "g":
            return T_SU3
        return np.ones((1, 1, 1), dtype=np.complex128)

    def _colour(self, tree, fixed=None, cache=None):
        """(legs, array) with axes legs + (open index,).  A leg in `fixed`
        (leg -> colour index) keeps only that colour (an axis of size 1);
        `cache` (a dict) shares subtrees between the terms of one pass."""
        if cache is not None and tree in cache:
            return cache[tree]
        if tree[0] == "L":
            d = self._colour_dim_leg(tree[1])
            e = np.eye(d, dtype=np.complex128)
            if fixed and tree[1] in fixed:
                e = e[[fixed[tree[1]]]]
            out = ((tree[1],), e)
            if cache is not None:
                cache[tree] = out
            return out
        _, kind, line, children, var = tree
        ch = [self._colour(c, fixed, cache) for c in children]
        legs = sum((c[0] for c in ch), ())
        ops = []
        # children: axes (legs..., X_i) with X_i = 40 + i; output label 45; e = 46
        for i, (cl, arr) in enumerate(ch):
            ops += [arr, list(cl) + [40 + i]]
        if kind in ("fin", "fout", "vec"):
            if kind == "vec":
                # children (column open l = 40, row open k = 41) -> adjoint out a = 45
                Tm = self._generators(line[1])
                ops += [Tm, [45, 41, 40]]
            else:
                # children (fermion open = 40, vector open a = 41)
                boson = BOSON_OF[line[1]]
                Tm = self._generators(boson)
                if kind == "fin":     # out k: T[a, k, l] psi_l
                    ops += [Tm, [41, 45, 40]]
                else:                 # out l: psibar_k T[a, k, l]
                    ops += [Tm, [41, 40, 45]]
        elif kind == "vvv":
            ops += [F_SU3, [40, 41, 45]]
        elif kind == "vvvv":
            ops += [F4_SU3[var - 1], [40, 41, 42, 45]]
        out = np.einsum(*ops, list(legs) + [45])
        if cache is not None:
            cache[tree] = (legs, out)
        return legs, out

    def _colour_columns(self, fixed=None):
        """[colours, t]: the colour factor of every term over the external
        colour assignments, the legs in `fixed` held at their colour (axes in
        leg order, flattened)."""
        cols = []
        cache = {} if fixed else None
        for t in self.terms:
            legs, arr = self._colour(t, fixed, cache)
            # open index = colour of the root leg
            order = list(legs) + [self.n - 1]
            arr = np.transpose(arr, np.argsort(order))
            cols.append(arr.reshape(-1))
        return np.stack(cols, axis=1)

    def colour_tensors(self):
        """C[colours, t]: the colour factor of every term over all external
        colour assignments (axes in leg order, flattened)."""
        if getattr(self, "_C", None) is None:
            self._C = self._colour_columns()
        return self._C

    # colour assignments x terms above which the colour matrix is summed in
    # chunks instead of from the whole colour tensor
    COLOUR_CHUNK = 1 << 26

    def colour_matrix(self):
        """G[t1, t2] = sum over all external colours of conj(c_t1) c_t2.
        For a process whose whole colour tensor is large (seven legs), the sum
        runs over chunks of colour assignments: the colours of the first
        gluon legs are held fixed in turn, and each chunk's C^dagger C is
        added; the colour tensor itself is never stored."""
        if self._G is None:
            dims = [self._colour_dim_leg(i) for i in range(self.n)]
            total = int(np.prod(dims)) * len(self.terms)
            if total <= self.COLOUR_CHUNK:
                C = self.colour_tensors()
                self._G = C.conj().T @ C
            else:
                gl = [i for i in range(self.n - 1) if dims[i] == 8]
                k = 0
                while total > self.COLOUR_CHUNK // 4 and k < len(gl):
                    total //= 8
                    k += 1
                chunks = [dict(zip(gl[:k], vals)) for vals in itertools.product(range(8), repeat=k)]
                workers = int(os.environ.get("MF_ORACLE_WORKERS", "0")) or (os.cpu_count() or 1)
                if workers > 1:
                    # chunks shared out over spawned processes (one numpy
                    # thread each); each returns the sum of its chunks
                    import multiprocessing as mp
                    parts = [chunks[w::workers] for w in range(workers)]
                    with mp.get_context("spawn").Pool(workers) as pool:
                        Gs = pool.map(_colour_gram_part, [(self, part) for part in parts if part])
                    self._G = np.sum(Gs, axis=0)
                else:
                    self._G = _colour_gram_part((self, chunks))
        return self._G

    # ---------------------------------------------------------------- leading colour
    def string_basis(self):
        """Colour strings: every pairing of the row-index quark legs (outgoing
        quarks, incoming antiquarks) with the column-index legs (incoming
        quarks, outgoing antiquarks), every distribution of the gluons over the
        strings and every order along each string; element
        prod_strings (T^{a_1} ... T^{a_m})_{row, col} over all external
        colours (axes in leg order, flattened), [colours, basis]."""
        if getattr(self, "_B", None) is not None:
            return self._B
        rows, cols, gluons = [], [], []
        for i, (part, inc) in enumerate(self.legs):
            kind, flav, _ = PARTICLES[part]
            if COLOUR_DIM[flav] == 8:
                gluons.append(i)
            elif COLOUR_DIM[flav] == 3:
                (rows if self.lines[i][2] == "out" else cols).append(i)
        dims = [self._colour_dim_leg(i) for i in range(self.n)]
        basis = []
        for perm in itertools.permutations(cols):
            for assign in itertools.product(range(len(rows)), repeat=len(gluons)):
                groups = [[g for g, s in zip(gluons, assign) if s == k] for k in range(len(rows))]
                for orders in itertools.product(*[list(itertools.permutations(gr)) for gr in groups]):
                    ops = []
                    for k, order in enumerate(orders):
                        r, c = rows[k], perm[k]
                        if not order:
                            ops += [np.eye(3), [r, c]]
                            continue
                        # chain T^{a_1}_{r x1} T^{a_2}_{x1 x2} ... T^{a_m}_{x_{m-1} c}
                        # (einsum labels: legs 0..n-1, chain indices from 10)
                        idx = [r] + [10 + 6 * k + j for j in range(len(order) - 1)] + [c]
                        for j, g in enumerate(order):
                            ops += [T_SU3, [g, idx[j], idx[j + 1]]]
                    out_axes = [i for i in range(self.n) if dims[i] > 1]
                    arr = np.einsum(*ops, out_axes) if ops else np.ones(())
                    basis.append(arr.reshape(-1))
        self._B = np.stack(basis, axis=1) if basis else np.ones((1, 1))
        return self._B

    def string_labels(self):
        """The strings of string_basis in its order: per basis element a tuple
        of (row leg, column leg, gluon legs in order along the string) per
        quark line."""
        rows, cols, gluons = [], [], []
        for i, (part, inc) in enumerate(self.legs):
            kind, flav, _ = PARTICLES[part]
            if COLOUR_DIM[flav] == 8:
                gluons.append(i)
            elif COLOUR_DIM[flav] == 3:
                (rows if self.lines[i][2] == "out" else cols).append(i)
        out = []
        for perm in itertools.permutations(cols):
            for assign in itertools.product(range(len(rows)), repeat=len(gluons)):
                groups = [[g for g, s in zip(gluons, assign) if s == k] for k in range(len(rows))]
                for orders in itertools.product(*[list(itertools.permutations(gr)) for gr in groups]):
                    out.append(tuple((rows[k], perm[k], tuple(orders[k])) for k in range(len(rows))))
        return out if out else [()]

    def leading_colour_weights(self, p):
        """Per point and string, sum over helicities of G_ss |A_s|^2 (the
        terms of msq_leading_colour), [N, basis]."""
        p = np.asarray(p, dtype=np.float64)
        B = self.string_basis()
        C = self.colour_tensors()
        P = np.linalg.pinv(B) @ C
        norms = np.real(np.sum(np.conj(B) * B, axis=0))
        cache = {}
        tot = np.zeros((B.shape[1], p.shape[0]))
        for hel in self.helicities():
            A = P @ self.amplitudes(p, hel, cache)
            tot += norms[:, None] * np.abs(A) ** 2
        return tot.T

    def colour_row_sums(self, p, k):
        """Per point i: sum over helicities of Re(conj(A_k) (G A)_k) with
        k = k[i], A the string coefficients of the colour-dressed amplitude
        and G = B^dagger B the strings' colour matrix (no averaging), [N]."""
        p = np.asarray(p, dtype=np.float64)
        k = np.asarray(k)
        B = self.string_basis()
        C = self.colour_tensors()
        P = np.linalg.pinv(B) @ C
        G = B.conj().T @ B
        cache = {}
        tot = np.zeros(p.shape[0])
        cols = np.arange(p.shape[0])
        for hel in self.helicities():
            A = P @ self.amplitudes(p, hel, cache)      # [basis, N]
            GA = G @ A
            tot += np.real(np.conj(A[k, cols]) * GA[k, cols])
        return tot

    def msq_leading_colour(self, p):
        """sum over helicities of sum_s G_ss |A_s|^2 (no averaging), with A the
        exact coefficients of the colour-dressed amplitude in the string basis
        and G_ss the basis elements' squared norms, [N]."""
        p = np.asarray(p, dtype=np.float64)
        B = self.string_basis()
        C = self.colour_tensors()
        P = np.linalg.pinv(B) @ C                      # terms -> string coefficients
        if np.max(np.abs(B @ P - C)) > 1e-12 * np.max(np.abs(C)):
            raise RuntimeError("colour factors outside the string basis")
        norms = np.real(np.sum(np.conj(B) * B, axis=0))
        cache = {}
        tot = np.zeros(p.shape[0])
        for hel in self.helicities():
            a = self.amplitudes(p, hel, cache)          # [T, N]
            A = P @ a                                   # [basis, N]
            tot += np.einsum("s,sn->n", norms, np.abs(A) ** 2)
        return tot

    # ---------------------------------------------------------------- kinematics
    def _sign(self, leg):
        return 1.0 if self.legs[leg][1] else -1.0

    def _P(self, tree, p):
        return sum(self._sign(l) * p[:, l] for l in self.legs_of(tree))

    def _mass(self, flav):
        m = self.masses.get(flav, 0.0)
        return m if hasattr(m, "d") else float(m)       # dual masses pass through

    def _coupling_ffv(self, flav):
        if BOSON_OF[flav] == "g":
            return 1j * self.g_s
        return 1j * self.e

    def _external(self, leg, lam, p, gauge_leg):
        part, inc = self.legs[leg]
        kind, flav, anti = PARTICLES[part]
        k = p[:, leg]
        if kind == "V":
            if leg == gauge_leg:
                return (k / k[:, 0:1]).astype(np.complex128)
            eps = polarisation(k, lam)
            return eps if inc else np.conj(eps)
        m = self._mass(flav)
        if not anti:
            u = spinor_u(k, m, lam)
            return u if inc else bar(u)
        v = spinor_v(k, m, lam)
        return bar(v) if inc else v

    def _kin(self, tree, hel, p, cache, gauge_leg, amputate=False):
        legs = self.legs_of(tree)
        key = (tree, tuple(hel[l] for l in legs), amputate)
        if key in cache:
            return cache[key]
        if tree[0] == "L":
            val = self._external(tree[1], hel[tree[1]], p, gauge_leg)
            cache[key] = val
            return val
        _, kind, line, children, var = tree
        vals = [self._kin(c, hel, p, cache, gauge_leg) for c in children]
        P = self._P(tree, p)
        if kind in ("fin", "fout"):
            flav = line[1]
            psi, J = vals
            cpl = self._coupling_ffv(flav)
            Js = slash(J)
            if kind == "fin":
                out = cpl * np.einsum("nij,nj->ni", Js, psi)
                q = P
            else:
                out = cpl * np.einsum("ni,nij->nj", psi, Js)
                q = -P
            if not amputate:
                m = self._mass(flav)
                S = 1j * (slash(q.astype(np.complex128)) + m * np.eye(4)[None]) \
                    / (mdot(q, q) - m * m)[:, None, None]
                if kind == "fin":
                    out = np.einsum("nij,nj->ni", S, out)
                else:
                    out = np.einsum("ni,nij->nj", out, S)
        elif kind == "vec":
            col, row = vals
            cpl = 1j * (self.g_s if line[1] == "g" else self.e)
            out = cpl * np.einsum("ni,mij,nj->nm", row, GAMMA, col)
            if not amputate:
                out = out * (-1j / mdot(P, P))[:, None]
        elif kind == "vvv":
            A, B = vals
            k1 = self._P(children[0], p)
            k2 = self._P(children[1], p)
            k3 = -(k1 + k2)
            out = self.g_s * (mdot(A, B)[:, None] * (k1 - k2)
                              + B * mdot(k2 - k3, A)[:, None]
                              + A * mdot(k3 - k1, B)[:, None])
            if not amputate:
                out = out * (-1j / mdot(P, P))[:, None]
        elif kind == "vvvv":
            A, B, C = vals
            if var == 1:
                t = mdot(A, C)[:, None] * B - mdot(B, C)[:, None] * A
            elif var == 2:
                t = mdot(A, B)[:, None] * C - mdot(B, C)[:, None] * A
            else:
                t = mdot(A, B)[:, None] * C - mdot(A, C)[:, None] * B
            out = -1j * self.g_s ** 2 * t
            if not amputate:
                out = out * (-1j / mdot(P, P))[:, None]
        else:
            raise ValueError(kind)
        cache[key] = out
        return out

    def amplitudes(self, p, hel, cache, gauge_leg=None):
        """Kinematic factor of every term for one helicity assignment, [T, N]."""
        root = self.n - 1
        wr = self._external(root, hel[root], p, gauge_leg)
        rl = self.lines[root]
        out = []
        for t in self.terms:
            top = self._kin(t, hel, p, cache, gauge_leg, amputate=True)
            if rl[0] == "V":
                out.append(mdot(top, wr))
            elif rl[2] == "in":          # root column spinor, top is a row
                out.append(np.einsum("ni,ni->n", top, wr))
            else:                        # root row spinor, top is a column
                out.append(np.einsum("ni,ni->n", wr, top))
        return np.stack(out)

    def helicities(self):
        return list(itertools.product((-1, 1), repeat=self.n))

    def msq_summed(self, p, gauge_leg=None, per_helicity=False):
        """sum over colours and helicities of |M|^2 (no averaging), [N]."""
        p = p if hasattr(p, "d") else np.asarray(p, dtype=np.float64)
        G = self.colour_matrix()
        cache = {}
        tot = np.zeros(p.shape[0])
        per = []
        for hel in self.helicities():
            a = self.amplitudes(p, hel, cache, gauge_leg)      # [T, N]
            val = np.real(np.einsum("tn,ts,sn->n", np.conj(a), G, a))
            tot = tot + val
            if per_helicity:
                per.append(val)
        return (tot, np.array(per)) if per_helicity else tot

    # ---------------------------------------------------------------- averages
    def average_factor(self):
        """1 / (initial spins x initial colours) x prod 1/k! for identical finals."""
        den = 1.0
        for part, inc in self.legs:
            if inc:
                kind, flav, _ = PARTICLES[part]
                den *= 2.0
                den *= COLOUR_DIM[flav]
        finals = [part for part, inc in self.legs if not inc]
        ident = 1.0
        for part in set(finals):
            ident /= math.factorial(finals.count(part))
        return ident / den

    def msq_avg(self, p, **kw):
        return self.msq_summed(p, **kw) * self.average_factor()
