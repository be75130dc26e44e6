"""Process builder: turns a 2 -> n process into the diagram program that
``mf_create_process`` consumes (the role MG5_aMC and the MadFlow exporter play
in Sec. 2.2 and Fig. 1 of the paper, written afresh for a small QCD/QED model).

Host-side, build-time Python.  It produces, for one process:

* the external legs (spin kind, fermion-flow role, mass);
* the diagram program: EXT ops (external wavefunctions), CUR ops (off-shell
  currents: each distinct sub-tree of the Feynman diagrams is computed once
  and shared by every diagram that contains it) and AMP ops (one per diagram,
  or three per four-gluon-vertex diagram, one per colour structure), each AMP
  op adding c * amplitude to one or more colour-flow amplitudes JAMP[k];
* the colour matrix C[k][l] = sum over colours of conj(B_k) B_l of the
  colour-flow basis B_k, as integer numerators over one denominator;
* the couplings of the Feynman rules (Peskin & Schroeder conventions):
  quark-gluon i g_s, lepton-photon i e, three-gluon g_s, four-gluon -i g_s^2;
* averaging factors and cut settings.

The colour decomposition is numerical: every diagram's colour tensor is
contracted from explicit SU(3) generators and projected onto the colour-flow
basis (products of open strings (t^a1 ... t^ak)_ij, one per quark line, over
all pairings of quark and antiquark indices); the projection is exact (the
residual is checked) and the coefficients are small rationals.
"""
from __future__ import annotations

import itertools
import json
import os
import math
from dataclasses import dataclass, field
from fractions import Fraction

import numpy as np

# routine ids: must match include/madflow_gb.h (enum mf_routine)
R_IXX, R_OXX, R_VXX = 0, 1, 2
R_FFV_AMP, R_FFV_FIN, R_FFV_FOUT, R_FFV_VEC = 10, 11, 12, 13
R_VVV_AMP, R_VVV_VEC = 20, 21
R_VVVV1_AMP, R_VVVV2_AMP, R_VVVV3_AMP = 30, 31, 32
R_VVVV1_VEC, R_VVVV2_VEC, R_VVVV3_VEC = 33, 34, 35

OP_EXT, OP_CUR, OP_AMP = 0, 1, 2

# external leg kinds (enum mf_leg_kind)
LEG_FERMION_IN, LEG_FERMION_OUT, LEG_VECTOR = 0, 1, 2

# particle table: name -> (spin, flavour, anti)
_PART = {
    "g": ("V", "g", False), "a": ("V", "a", False),
    "u": ("F", "u", False), "u~": ("F", "u", True),
    "t": ("F", "t", False), "t~": ("F", "t", True),
    "e-": ("F", "e", False), "e+": ("F", "e", True),
    "mu-": ("F", "mu", False), "mu+": ("F", "mu", True),
}
_GAUGE = {"u": "g", "t": "g", "e": "a", "mu": "a"}
_NCOL = {"g": 8, "a": 1, "u": 3, "t": 3, "e": 1, "mu": 1}


def _su3():
    lam = np.zeros((8, 3, 3), dtype=complex)
    # Gell-Mann matrices
    lam[0][[0, 1], [1, 0]] = 1
    lam[1][0, 1], lam[1][1, 0] = -1j, 1j
    lam[2][0, 0], lam[2][1, 1] = 1, -1
    lam[3][[0, 2], [2, 0]] = 1
    lam[4][0, 2], lam[4][2, 0] = -1j, 1j
    lam[5][[1, 2], [2, 1]] = 1
    lam[6][1, 2], lam[6][2, 1] = -1j, 1j
    lam[7] = np.diag([1, 1, -2]) / math.sqrt(3)
    t = lam / 2
    # [t^a, t^b] = i f^abc t^c  ->  f^abc = -2 i Tr([t^a, t^b] t^c)
    comm = np.einsum("aij,bjk->abik", t, t) - np.einsum("bij,ajk->abik", t, t)
    f = np.real(-2j * np.einsum("abik,cki->abc", comm, t))
    return t, f


T_GEN, F_ABC = _su3()


# ---------------------------------------------------------------------------
# topology: every tree with the model's vertices, sharing common sub-trees
# ---------------------------------------------------------------------------
@dataclass(frozen=True)
class Node:
    kind: str            # 'ext', 'fin', 'fout', 'vec', 'vvv', 'vvvv'
    line: tuple          # ('F', flavour, 'in'|'out') or ('V', boson)
    children: tuple = () # Node tuple
    leg: int = -1        # for 'ext'
    variant: int = 0     # four-gluon colour structure 1..3

    @property
    def legs(self):
        if self.kind == "ext":
            return frozenset((self.leg,))
        s = frozenset()
        for c in self.children:
            s = s | c.legs
        return s


def _leg_line(particle, incoming):
    spin, flav, anti = _PART[particle]
    if spin == "V":
        return ("V", flav)
    column = incoming != anti     # u of incoming particle, v of outgoing antiparticle
    return ("F", flav, "in" if column else "out")


class Topology:
    def __init__(self, legs):
        self.legs = legs
        self.lines = [_leg_line(p, i) for p, i in legs]
        self.flavours = sorted({_PART[p][1] for p, _ in legs if _PART[p][0] == "F"})
        self.cache = {}

    def subtrees(self, S, line):
        key = (S, line)
        if key in self.cache:
            return self.cache[key]
        res = []
        if len(S) == 1:
            leg = next(iter(S))
            if self.lines[leg] == line:
                res.append(Node("ext", line, leg=leg))
        elif line[0] == "F":
            gauge = _GAUGE[line[1]]
            kind = "fin" if line[2] == "in" else "fout"
            for A, B in self._ordered_pairs(S):
                for f in self.subtrees(A, line):
                    for v in self.subtrees(B, ("V", gauge)):
                        res.append(Node(kind, line, (f, v)))
        else:
            boson = line[1]
            for flav in self.flavours:
                if _GAUGE[flav] != boson:
                    continue
                for A, B in self._ordered_pairs(S):
                    for c in self.subtrees(A, ("F", flav, "in")):
                        for r in self.subtrees(B, ("F", flav, "out")):
                            res.append(Node("vec", line, (c, r)))
            if boson == "g":
                for A, B in self._set_partitions(S, 2):
                    for a in self.subtrees(A, line):
                        for b in self.subtrees(B, line):
                            res.append(Node("vvv", line, (a, b)))
                for A, B, C in self._set_partitions(S, 3):
                    for a in self.subtrees(A, line):
                        for b in self.subtrees(B, line):
                            for c in self.subtrees(C, line):
                                for v in (1, 2, 3):
                                    res.append(Node("vvvv", line, (a, b, c), variant=v))
        self.cache[key] = res
        return res

    @staticmethod
    def _ordered_pairs(S):
        items = sorted(S)
        for r in range(1, len(items)):
            for A in itertools.combinations(items, r):
                A = frozenset(A)
                yield A, S - A

    @staticmethod
    def _set_partitions(S, k):
        """Unordered partitions of S into k non-empty blocks (blocks ordered by
        their smallest element)."""
        items = sorted(S)

        def rec(rest, blocks):
            if not rest:
                if len(blocks) == k:
                    yield tuple(frozenset(b) for b in blocks)
                return
            x, tail = rest[0], rest[1:]
            for b in blocks:
                b.append(x)
                yield from rec(tail, blocks)
                b.pop()
            if len(blocks) < k:
                blocks.append([x])
                yield from rec(tail, blocks)
                blocks.pop()
        yield from rec(items, [])


# ---------------------------------------------------------------------------
# colour: explicit tensors, projected onto the colour-flow basis
# ---------------------------------------------------------------------------
class ColourSpace:
    """Tensor over the external colour indices, axes in leg order."""

    def __init__(self, legs):
        self.legs = legs
        self.dims = [_NCOL[_PART[p][1]] for p, _ in legs]

    def node_tensor(self, node: Node):
        """(legs tuple, array[..., open])."""
        if node.kind == "ext":
            d = self.dims[node.leg]
            return (node.leg,), np.eye(d, dtype=complex)
        parts = [self.node_tensor(c) for c in node.children]
        legs = tuple(l for p in parts for l in p[0])
        args = []
        for k, (lg, arr) in enumerate(parts):
            args += [arr, list(lg) + [20 + k]]
        if node.kind in ("fin", "fout", "vec"):
            boson = node.line[1] if node.kind == "vec" else _GAUGE[node.line[1]]
            gen = T_GEN if boson == "g" else np.ones((1, 1, 1), dtype=complex)
            if node.kind == "fin":       # (col open l=20, vec a=21) -> k
                args += [gen, [21, 30, 20]]
            elif node.kind == "fout":    # (row open k=20, vec a=21) -> l
                args += [gen, [21, 20, 30]]
            else:                        # (col l=20, row k=21) -> a
                args += [gen, [30, 21, 20]]
        elif node.kind == "vvv":
            args += [F_ABC, [20, 21, 30]]
        else:
            f4 = {1: "abe,cde->abcd", 2: "ace,bde->abcd", 3: "ade,bce->abcd"}[node.variant]
            args += [np.einsum(f4, F_ABC, F_ABC), [20, 21, 22, 30]]
        out = np.einsum(*args, list(legs) + [30])
        return legs, out

    def full(self, node: Node, root: int):
        legs, arr = self.node_tensor(node)
        order = list(legs) + [root]
        return np.transpose(arr, np.argsort(order))

    def flow_basis(self):
        """Colour-flow basis tensors [n_basis, prod(dims)] and their labels."""
        outs, ins, gluons = [], [], []
        for i, (p, inc) in enumerate(self.legs):
            spin, flav, anti = _PART[p]
            if flav == "g":
                gluons.append(i)
            elif _NCOL[flav] == 3:
                # fundamental 'out' index: outgoing quark or incoming antiquark
                (outs if (not inc) != anti else ins).append(i)
        nq = len(outs)
        basis, labels = [], []
        for perm in itertools.permutations(ins):
            for assign in itertools.product(range(max(nq, 1)), repeat=len(gluons)):
                groups = [[g for g, a in zip(gluons, assign) if a == s] for s in range(nq)]
                for orders in itertools.product(*[list(itertools.permutations(g)) for g in groups]):
                    t = np.ones(self.dims, dtype=complex)
                    for s in range(nq):
                        t = t * self._string(outs[s], perm[s], orders[s])
                    basis.append(t.reshape(-1))
                    labels.append(tuple((outs[s], perm[s], orders[s]) for s in range(nq)))
        B = np.stack(basis, axis=1) if basis else np.ones((int(np.prod(self.dims)), 1), dtype=complex)
        if not basis:
            labels = [()]
        return B, labels

    def _string(self, i_out, j_in, gl):
        """(t^gl0 ... t^glk)_{i_out j_in} broadcast to the full index space."""
        n = len(self.legs)
        if not gl:
            m = np.eye(3, dtype=complex)
            shape = [1] * n
            shape[i_out], shape[j_in] = 3, 3
            return m.reshape(shape) if i_out < j_in else m.T.reshape(shape)
        letters = "abcdefgh"
        expr = ",".join(f"{letters[k]}{'pqrstuvw'[k]}{'pqrstuvw'[k + 1]}" for k in range(len(gl)))
        out = "".join(letters[k] for k in range(len(gl))) + "p" + "pqrstuvw"[len(gl)]
        arr = np.einsum(expr + "->" + out, *([T_GEN] * len(gl)))
        axes = list(gl) + [i_out, j_in]
        shape = [1] * n
        for ax, d in zip(axes, arr.shape):
            shape[ax] = d
        perm = np.argsort(axes)
        return np.transpose(arr, perm).reshape(shape)


def _rationalise(x, max_den=64, tol=1e-9):
    f = Fraction(x).limit_denominator(max_den)
    if abs(float(f) - x) > tol * max(1.0, abs(x)):
        raise ValueError(f"colour coefficient {x} is not a small rational")
    return f


# ---------------------------------------------------------------------------
# the program
# ---------------------------------------------------------------------------
@dataclass
class Op:
    kind: int
    routine: int
    inputs: tuple = ()
    leg: int = -1
    coupling: int = -1
    mass: float = 0.0
    width: float = 0.0
    terms: list = field(default_factory=list)   # [(jamp, re, im)]


@dataclass
class ProcessProgram:
    name: str
    legs: list                 # [(particle, incoming)]
    leg_kind: list
    leg_mass: list
    ops: list
    couplings: list            # complex
    colour_num: np.ndarray     # int [nc, nc]
    colour_den: int
    n_diagrams: int
    average: float             # 1/(spins x colours) x identical-particle factor
    alpha_s_power: int
    basis_labels: list


# Programs whose construction takes minutes (gg -> tt~ggg: 1240 diagrams, a
# 120-flow colour basis) are stored once as JSON under programs/ by
# programs/store_programs.py; build_program loads a stored structure when
# one exists for the same name and legs and fills in the masses and
# couplings of the call.
PROGRAM_STORE = os.path.join(os.path.dirname(os.path.abspath(__file__)), "programs")


def _couplings(alpha_s, alpha):
    g_s = math.sqrt(4 * math.pi * alpha_s)
    e = math.sqrt(4 * math.pi * alpha)
    return [1j * g_s, 1j * e, g_s + 0j, -1j * g_s * g_s]


def store_program(prog: "ProcessProgram", masses: dict, path: str):
    """Write the structure of a program (masses as flavour names) to JSON."""
    inv = {}
    for flav, m in masses.items():
        inv.setdefault(float(m), flav)

    def flav_of(m):
        return "" if m == 0.0 else inv[float(m)]
    rec = {"name": prog.name, "legs": [[p, bool(i)] for p, i in prog.legs], "leg_kind": list(prog.leg_kind),
           "leg_mass": [flav_of(m) for m in prog.leg_mass],
           "ops": [[o.kind, o.routine, list(o.inputs), o.leg, o.coupling, flav_of(o.mass),
                    [[k, re, im] for k, re, im in o.terms]] for o in prog.ops],
           "colour_num": prog.colour_num.tolist(), "colour_den": int(prog.colour_den),
           "n_diagrams": prog.n_diagrams, "average": prog.average, "alpha_s_power": prog.alpha_s_power,
           "basis_labels": [[[r, c, list(g)] for r, c, g in label] for label in prog.basis_labels]}
    with open(path, "w") as fh:
        json.dump(rec, fh, separators=(",", ":"))


def _stored_program(name, legs, masses, alpha_s, alpha):
    path = os.path.join(PROGRAM_STORE, name + ".json")
    if not os.path.exists(path):
        return None
    with open(path) as fh:
        rec = json.load(fh)
    if [(p, bool(i)) for p, i in rec["legs"]] != legs:
        return None

    def mass(flav):
        return float(masses.get(flav, 0.0)) if flav else 0.0
    ops = [Op(k, r, tuple(ins), leg=leg, coupling=c, mass=mass(mf), terms=[tuple(t) for t in terms])
           for k, r, ins, leg, c, mf, terms in rec["ops"]]
    labels = [tuple((r, c, tuple(g)) for r, c, g in label) for label in rec["basis_labels"]]
    return ProcessProgram(rec["name"], legs, rec["leg_kind"], [mass(f) for f in rec["leg_mass"]], ops,
                          _couplings(alpha_s, alpha), np.array(rec["colour_num"], dtype=np.int64),
                          rec["colour_den"], rec["n_diagrams"], rec["average"], rec["alpha_s_power"], labels)


def build_program(name, legs, masses, alpha_s, alpha):
    """legs: [(particle, incoming)], incoming first. masses: flavour -> mass."""
    legs = [(p, bool(i)) for p, i in legs]
    stored = _stored_program(name, legs, masses, alpha_s, alpha)
    if stored is not None:
        return stored
    n = len(legs)
    topo = Topology(legs)
    lines = topo.lines
    # root: the last leg that is a fermion (so one-quark-line processes never
    # need a gluon produced from the whole quark line), else the last leg
    fermions = [i for i in range(n) if lines[i][0] == "F"]
    root = fermions[-1] if fermions else n - 1
    rest = frozenset(range(n)) - {root}
    need = lines[root] if lines[root][0] == "V" else ("F", lines[root][1],
                                                      "out" if lines[root][2] == "in" else "in")
    tops = [t for t in topo.subtrees(rest, need) if t.kind != "ext"]
    # diagrams (a four-gluon vertex's three colour structures are one diagram)
    def strip(t):
        return Node(t.kind, t.line, tuple(strip(c) for c in t.children), t.leg, 0)
    n_diagrams = len({strip(t) for t in tops})

    couplings = _couplings(alpha_s, alpha)
    C_FFV_G, C_FFV_A, C_VVV, C_VVVV = 0, 1, 2, 3

    def mass_of(line):
        return float(masses.get(line[1], 0.0)) if line[0] == "F" else 0.0

    ops = []
    slot = {}
    leg_kind, leg_mass = [], []
    for i, (p, inc) in enumerate(legs):
        ln = lines[i]
        if ln[0] == "V":
            k, r = LEG_VECTOR, R_VXX
        elif ln[2] == "in":
            k, r = LEG_FERMION_IN, R_IXX
        else:
            k, r = LEG_FERMION_OUT, R_OXX
        leg_kind.append(k)
        leg_mass.append(mass_of(ln))
        ops.append(Op(OP_EXT, r, leg=i))
        slot[Node("ext", ln, leg=i)] = i

    def emit(node):
        if node in slot:
            return slot[node]
        ins = tuple(emit(c) for c in node.children)
        m = mass_of(node.line)
        if node.kind == "fin":
            op = Op(OP_CUR, R_FFV_FIN, ins, coupling=C_FFV_G if _GAUGE[node.line[1]] == "g" else C_FFV_A, mass=m)
        elif node.kind == "fout":
            op = Op(OP_CUR, R_FFV_FOUT, ins, coupling=C_FFV_G if _GAUGE[node.line[1]] == "g" else C_FFV_A, mass=m)
        elif node.kind == "vec":
            # inputs ordered (row, column) for the routine
            op = Op(OP_CUR, R_FFV_VEC, (ins[1], ins[0]), coupling=C_FFV_G if node.line[1] == "g" else C_FFV_A)
        elif node.kind == "vvv":
            op = Op(OP_CUR, R_VVV_VEC, ins, coupling=C_VVV)
        else:
            op = Op(OP_CUR, (R_VVVV1_VEC, R_VVVV2_VEC, R_VVVV3_VEC)[node.variant - 1], ins, coupling=C_VVVV)
        ops.append(op)
        slot[node] = len(ops) - 1
        return slot[node]

    # colour decomposition of every amplitude term
    cs = ColourSpace(legs)
    B, labels = cs.flow_basis()
    # keep an independent subset of the basis
    q, rmat = np.linalg.qr(B)
    keep = [k for k in range(B.shape[1]) if abs(rmat[k, k]) > 1e-9]
    B = B[:, keep]
    labels = [labels[k] for k in keep]
    pinv = np.linalg.pinv(B)

    amp_ops = []
    for t in tops:
        ins = [emit(c) for c in t.children]
        r_slot = root
        if t.kind == "fout":      # row from (row, vec) + root column
            op = Op(OP_AMP, R_FFV_AMP, (ins[0], r_slot, ins[1]),
                    coupling=C_FFV_G if _GAUGE[t.line[1]] == "g" else C_FFV_A)
        elif t.kind == "fin":     # column from (column, vec) + root row
            op = Op(OP_AMP, R_FFV_AMP, (r_slot, ins[0], ins[1]),
                    coupling=C_FFV_G if _GAUGE[t.line[1]] == "g" else C_FFV_A)
        elif t.kind == "vec":     # (column, row) + root vector
            op = Op(OP_AMP, R_FFV_AMP, (ins[1], ins[0], r_slot),
                    coupling=C_FFV_G if t.line[1] == "g" else C_FFV_A)
        elif t.kind == "vvv":
            op = Op(OP_AMP, R_VVV_AMP, (ins[0], ins[1], r_slot), coupling=C_VVV)
        else:
            op = Op(OP_AMP, (R_VVVV1_AMP, R_VVVV2_AMP, R_VVVV3_AMP)[t.variant - 1],
                    (ins[0], ins[1], ins[2], r_slot), coupling=C_VVVV)
        D = cs.full(t, root).reshape(-1)
        c = pinv @ D
        resid = np.max(np.abs(B @ c - D)) if D.size else 0.0
        if resid > 1e-10:
            raise RuntimeError(f"colour projection failed for {name}: residual {resid}")
        for k, ck in enumerate(c):
            if abs(ck) > 1e-12:
                re = float(_rationalise(ck.real)) if abs(ck.real) > 1e-12 else 0.0
                im = float(_rationalise(ck.imag)) if abs(ck.imag) > 1e-12 else 0.0
                op.terms.append((k, re, im))
        amp_ops.append(op)
    ops.extend(amp_ops)

    # colour matrix as integer numerators over a common denominator
    Cm = B.conj().T @ B
    if np.max(np.abs(Cm.imag)) > 1e-10:
        raise RuntimeError("colour matrix is not real")
    Cr = Cm.real
    den = None
    for d in range(1, 1000):
        if np.max(np.abs(Cr * d - np.round(Cr * d))) < 1e-8:
            den = d
            break
    if den is None:
        raise RuntimeError("colour matrix is not rational with a small denominator")
    num = np.round(Cr * den).astype(np.int64)

    # averages: spins (2 per incoming particle) x colours, identical finals
    avg = 1.0
    for p, inc in legs:
        if inc:
            avg /= 2.0 * _NCOL[_PART[p][1]]
    finals = [p for p, inc in legs if not inc]
    for p in set(finals):
        avg /= math.factorial(finals.count(p))
    # alpha_s power: a pure-QCD tree amplitude with n legs carries g_s^(n-2)
    qcd = all(_PART[p][1] in ("g", "u", "t") for p, _ in legs)
    k_as = (n - 2) if qcd else 0
    return ProcessProgram(name, legs, leg_kind, leg_mass, ops, couplings, num, den,
                          n_diagrams, avg, k_as, labels)


def lhe_colour_tags(prog: ProcessProgram) -> np.ndarray:
    """Les Houches colour and anticolour tags of every colour flow of the
    program, [n_flows, n_legs, 2] (the flow order of the colour basis).

    A flow is a product of open strings (t^g1 ... t^gk)_{row, column}.  Along
    a string the colour line of the row quark (an outgoing quark, or an
    incoming antiquark) passes each gluon in turn -- the gluon absorbs it as
    its anticolour and emits a new line as its colour -- and ends as the
    anticolour of the column quark (an outgoing antiquark or an incoming
    quark); these are the all-outgoing assignments, and an incoming particle
    carries them swapped.  Lines are numbered from 501."""
    n = len(prog.legs)
    tags = np.zeros((len(prog.basis_labels), n, 2), dtype=np.int32)
    for k, label in enumerate(prog.basis_labels):
        line = 500
        c = {}
        for row, col, gluons in label:
            line += 1
            c[(row, 0)] = line
            for g in gluons:
                c[(g, 1)] = line
                line += 1
                c[(g, 0)] = line
            c[(col, 1)] = line
        for i, (_, incoming) in enumerate(prog.legs):
            colour, anticolour = c.get((i, 0), 0), c.get((i, 1), 0)
            tags[k, i] = (anticolour, colour) if incoming else (colour, anticolour)
    return tags


def helicity_table(n_legs):
    return [list(h) for h in itertools.product((-1, 1), repeat=n_legs)]
