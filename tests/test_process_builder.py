"""Host-side checks of the process builder (CPU only).

The builder's diagram program (shared currents, colour-flow coefficients,
colour matrix) is run through a small numpy interpreter of the routine
semantics declared in include/madflow_gb.h and compared with the oracle's
brute-force |M|^2.  This validates the program the CUDA library compiles,
independently of any GPU.
"""
import math

import numpy as np
import pytest

import workloads as W
from oracle.feynman import GAMMA, bar, mdot, polarisation, slash, spinor_u, spinor_v
from oracle.integrand import Integrand
from paper_2106_10279_gb300 import process as P


def _run_program(prog, p, hel):
    """Colour-flow amplitudes JAMP for one helicity, [nc, N]."""
    N = p.shape[0]
    wf, mom = [], []
    nc = prog.colour_num.shape[0]
    jamp = np.zeros((nc, N), dtype=complex)
    cpl = prog.couplings
    for op in prog.ops:
        if op.kind == P.OP_EXT:
            leg = op.leg
            part, inc = prog.legs[leg]
            k = p[:, leg]
            lam = hel[leg]
            m = prog.leg_mass[leg]
            anti = part.endswith("~") or part.endswith("+")
            if op.routine == P.R_VXX:
                e = polarisation(k, lam)
                v = e if inc else np.conj(e)
            elif op.routine == P.R_IXX:
                v = spinor_v(k, m, lam) if anti else spinor_u(k, m, lam)
            else:
                v = bar(spinor_v(k, m, lam)) if anti else bar(spinor_u(k, m, lam))
            wf.append(v)
            mom.append(k if inc else -k)
            continue
        ins = [wf[i] for i in op.inputs]
        pin = [mom[i] for i in op.inputs]
        g = cpl[op.coupling]
        if op.kind == P.OP_CUR:
            Pc = sum(pin)
            r = op.routine
            if r in (P.R_FFV_FIN, P.R_FFV_FOUT):
                psi, V = ins
                q = Pc if r == P.R_FFV_FIN else -Pc
                S = 1j * (slash(q.astype(complex)) + op.mass * np.eye(4)[None]) / (mdot(q, q) - op.mass ** 2)[:, None, None]
                if r == P.R_FFV_FIN:
                    out = np.einsum("nij,nj->ni", S, g * np.einsum("nij,nj->ni", slash(V), psi))
                else:
                    out = np.einsum("ni,nij->nj", g * np.einsum("ni,nij->nj", psi, slash(V)), S)
            elif r == P.R_FFV_VEC:
                row, col = ins
                out = -1j / mdot(Pc, Pc)[:, None] * g * np.einsum("ni,mij,nj->nm", row, GAMMA, col)
            elif r == P.R_VVV_VEC:
                A, B = ins
                k1, k2 = pin
                k3 = -(k1 + k2)
                out = -1j / mdot(Pc, Pc)[:, None] * g * (mdot(A, B)[:, None] * (k1 - k2)
                                                         + B * mdot(k2 - k3, A)[:, None]
                                                         + A * mdot(k3 - k1, B)[:, None])
            else:
                A, B, C = ins
                s = r - P.R_VVVV1_VEC + 1
                t = {1: mdot(A, C)[:, None] * B - mdot(B, C)[:, None] * A,
                     2: mdot(A, B)[:, None] * C - mdot(B, C)[:, None] * A,
                     3: mdot(A, B)[:, None] * C - mdot(A, C)[:, None] * B}[s]
                out = -1j / mdot(Pc, Pc)[:, None] * g * t
            wf.append(out)
            mom.append(Pc)
        else:
            r = op.routine
            if r == P.R_FFV_AMP:
                row, col, V = ins
                amp = g * np.einsum("ni,nij,nj->n", row, slash(V), col)
            elif r == P.R_VVV_AMP:
                A, B, C = ins
                k1, k2, k3 = pin
                amp = g * (mdot(A, B) * mdot(k1 - k2, C) + mdot(B, C) * mdot(k2 - k3, A)
                           + mdot(C, A) * mdot(k3 - k1, B))
            else:
                A, B, C, D = ins
                s = r - P.R_VVVV1_AMP + 1
                amp = g * {1: mdot(A, C) * mdot(B, D) - mdot(A, D) * mdot(B, C),
                           2: mdot(A, B) * mdot(C, D) - mdot(A, D) * mdot(B, C),
                           3: mdot(A, B) * mdot(C, D) - mdot(A, C) * mdot(B, D)}[s]
            for k, re, im in op.terms:
                jamp[k] += (re + 1j * im) * amp
            wf.append(None)
            mom.append(None)
    return jamp


def _program_msq(prog, p):
    C = prog.colour_num / prog.colour_den
    tot = np.zeros(p.shape[0])
    for hel in P.helicity_table(len(prog.legs)):
        J = _run_program(prog, p, hel)
        tot += np.real(np.einsum("kn,kl,ln->n", np.conj(J), C, J))
    return tot * prog.average


@pytest.fixture(scope="module")
def programs():
    out = {}
    for name, wl in W.WORKLOADS.items():
        out[name] = P.build_program(name, [(l.particle, l.incoming) for l in wl.legs],
                                    {"t": wl.m_top}, wl.alpha_s, wl.alpha)
    return out


def test_diagram_counts_and_colour_dimensions(programs):
    exp = {"ee_mumu": (1, 1), "gg_ttx": (3, 2), "uux_ttx": (1, 2), "gg_ttxg": (16, 6),
           "uux_ttxg": (5, 4), "gg_ttxgg": (123, 24)}
    for name, (nd, nc) in exp.items():
        assert programs[name].n_diagrams == nd
        assert programs[name].colour_num.shape == (nc, nc)
    assert programs["gg_ttx"].colour_den == 3
    assert programs["gg_ttxg"].colour_den == 9
    assert programs["gg_ttxgg"].colour_den == 54


def test_colour_matrices_positive_definite(programs):
    for prog in programs.values():
        C = prog.colour_num / prog.colour_den
        assert np.allclose(C, C.T)
        assert np.min(np.linalg.eigvalsh(C)) > 0


@pytest.mark.parametrize("name,n", [("ee_mumu", 50), ("gg_ttx", 50), ("uux_ttx", 50),
                                    ("gg_ttxg", 20), ("uux_ttxg", 20), ("gg_ttxgg", 6)])
def test_program_reproduces_oracle_msq(name, n, programs, oracle_processes):
    wl = W.WORKLOADS[name]
    proc = oracle_processes(name)
    I = Integrand(wl, process=proc)
    x = W.uniform_points(wl.ndim, n, 17)
    p, *_ = I.kinematics(x)
    ref = proc.msq_avg(p)
    got = _program_msq(programs[name], p)
    assert np.max(np.abs(got / ref - 1)) < 1e-12


@pytest.mark.parametrize("name", ["ee_mumu", "gg_ttx", "uux_ttx", "gg_ttxg", "uux_ttxg", "gg_ttxgg"])
def test_lhe_colour_tags_agree_with_the_oracle(name):
    # the builder's tags per colour flow against the oracle's, written
    # independently from each side's own string labels (same basis order:
    # the basis tensors are compared element by element first)
    from paper_2106_10279_gb300 import api
    from paper_2106_10279_gb300.process import ColourSpace, lhe_colour_tags
    from oracle.integrand import oracle_process
    from oracle.unweight import colour_tags
    wl = W.WORKLOADS[name]
    d = api.descriptor_for_workload(wl)
    op = oracle_process(wl)
    B, _ = ColourSpace(d.prog.legs).flow_basis()
    assert np.array_equal(B, op.string_basis())
    assert np.array_equal(lhe_colour_tags(d.prog), colour_tags(op.string_labels(), op.legs))
