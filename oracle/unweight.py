"""Unweighting and event records of the oracle (Sec. 2.5 of the MadFlow
paper: weighted Vegas points are turned into unweighted events written to
Les Houches Event files).  Test infrastructure only.

Definitions (hit-or-miss unweighting against a maximum weight w_max):

* point i with weight w_i is kept when |w_i| > u_i w_max, with u_i a unit
  number drawn independently of the point (here the first word of the Philox
  counter (i, iteration, subprocess, 15), mapped like every other unit number);
* a kept point carries the event weight sign(w_i) max(|w_i|, w_max) / N, so
  that the expected sum of the event weights equals (1/N) sum_i w_i, the
  integral estimate (points above w_max are kept with their own weight);
* the momenta of an event are those of the partonic centre-of-mass frame
  boosted along the beam axis by the rapidity y = (ln x1 - ln x2) / 2 of the
  parton pair, so that the incoming partons carry x1 and x2 of the beam
  energies;
* a kept event gets a colour flow: the string s of the colour basis is
  drawn with probability proportional to its leading-colour weight (the
  helicity sum of |A_s|^2 times the string's squared norm), by the first
  unit number of Philox counter (i, iteration, subprocess, 13): the first
  string, in basis order, whose cumulative weight exceeds u times the total;
* its colour tags follow the string: the row quark's colour line runs
  through the gluons in string order (each gluon takes the line as its
  anticolour and starts a new line as its colour) into the column quark's
  anticolour, all particles taken as outgoing; an incoming particle then
  swaps colour and anticolour; lines are numbered from 501 in that order.
"""
from __future__ import annotations

import numpy as np

from oracle.philox import philox4x64_10, to_unit

UNWEIGHT_BLOCK = 15
COLOUR_BLOCK = 13


def accept_uniforms(seed: int, iteration: int, subprocess: int, n: int) -> np.ndarray:
    """The accept/reject unit numbers of points 0 .. n-1."""
    ctr = np.zeros((n, 4), dtype=np.uint64)
    ctr[:, 0] = np.arange(n, dtype=np.uint64)
    ctr[:, 1] = np.uint64(iteration)
    ctr[:, 2] = np.uint64(subprocess)
    ctr[:, 3] = np.uint64(UNWEIGHT_BLOCK)
    words = philox4x64_10(ctr, np.array([seed, 0], dtype=np.uint64))
    return to_unit(words[:, 0])


def keep(w: np.ndarray, u: np.ndarray, w_max: float) -> np.ndarray:
    return np.abs(w) > u * w_max


def event_weights(w: np.ndarray, w_max: float, n_points: int) -> np.ndarray:
    return np.sign(w) * np.maximum(np.abs(w), w_max) / n_points


def boost_z(p: np.ndarray, y: np.ndarray) -> np.ndarray:
    """Boost momenta p [N, n, 4] (E, px, py, pz) along z by rapidity y [N]."""
    ch, sh = np.cosh(y)[:, None], np.sinh(y)[:, None]
    out = p.copy()
    out[:, :, 0] = ch * p[:, :, 0] + sh * p[:, :, 3]
    out[:, :, 3] = sh * p[:, :, 0] + ch * p[:, :, 3]
    return out


def lab_frame(p_cm: np.ndarray, x1: np.ndarray, x2: np.ndarray) -> np.ndarray:
    return boost_z(p_cm, 0.5 * (np.log(x1) - np.log(x2)))


def colour_uniforms(seed: int, iteration: int, subprocess: int, idx: np.ndarray) -> np.ndarray:
    """The colour-flow unit numbers of points idx."""
    idx = np.asarray(idx, dtype=np.uint64)
    ctr = np.zeros((idx.size, 4), dtype=np.uint64)
    ctr[:, 0] = idx
    ctr[:, 1] = np.uint64(iteration)
    ctr[:, 2] = np.uint64(subprocess)
    ctr[:, 3] = np.uint64(COLOUR_BLOCK)
    words = philox4x64_10(ctr, np.array([seed, 0], dtype=np.uint64))
    return to_unit(words[:, 0])


def draw_flows(weights: np.ndarray, u: np.ndarray):
    """Index of the drawn string per point (weights [N, basis]) and the
    distance of u times the total from the nearest cumulative boundary,
    relative to the total (how close the draw was to a tie)."""
    cum = np.cumsum(weights, axis=1)
    tot = cum[:, -1]
    target = u * tot
    pick = np.argmax((cum > target[:, None]) & (weights > 0), axis=1)
    gap = np.min(np.abs(cum - target[:, None]), axis=1) / np.where(tot > 0, tot, 1.0)
    return pick, gap


def colour_tags(labels, legs) -> np.ndarray:
    """LHE (colour, anticolour) per string label and leg, [basis, n_legs, 2]."""
    n = len(legs)
    out = np.zeros((len(labels), n, 2), dtype=np.int64)
    for k, label in enumerate(labels):
        col = [0] * n
        anti = [0] * n
        line = 500
        for row, column, gluons in label:
            line += 1
            col[row] = line
            for g in gluons:
                anti[g] = line
                line += 1
                col[g] = line
            anti[column] = line
        for i, (_, incoming) in enumerate(legs):
            out[k, i] = (anti[i], col[i]) if incoming else (col[i], anti[i])
    return out
