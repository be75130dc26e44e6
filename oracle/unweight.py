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
  energies.
"""
from __future__ import annotations

import numpy as np

from oracle.philox import philox4x64_10, to_unit

UNWEIGHT_BLOCK = 15


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
