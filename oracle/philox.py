"""Philox4x64-10 counter-based generator, written from its published
definition (J. Salmon, M. Moraes, R. Dror, D. Shaw, "Parallel random numbers:
as easy as 1, 2, 3", SC'11, Sec. 3-4), vectorised over counters with numpy.

The Vegas iteration (Sec. 2.2 of the MadFlow paper: "generation of random
numbers, computation of the phase space kinematics, matrix element evaluation
and histogram accumulation") draws its uniforms from this generator:

    key     = (seed, 0)
    counter = (event index, iteration index, subprocess index, dimension block)
    u       = ((r >> 11) | 1) * 2^-53           (odd multiples of 2^-53: in (0,1))

Dimension j of an event uses word j % 4 of the block j // 4.

Pinned in tests against ``numpy.random.Philox`` (an independent library
implementation of the same bijection) and by output uniformity checks.
"""
from __future__ import annotations

import numpy as np

M0 = np.uint64(0xD2E7470EE14C6C93)
M1 = np.uint64(0xCA5A826395121157)
W0 = np.uint64(0x9E3779B97F4A7C15)   # golden ratio
W1 = np.uint64(0xBB67AE8584CAA73B)   # sqrt(3) - 1
_MASK32 = np.uint64(0xFFFFFFFF)
_S32 = np.uint64(32)


def _mulhilo(a: np.uint64, b: np.ndarray):
    """Full 64x64 -> 128-bit product as (hi, lo), exact, by 32-bit limbs."""
    b = b.astype(np.uint64)
    a_lo, a_hi = a & _MASK32, a >> _S32
    b_lo, b_hi = b & _MASK32, b >> _S32
    ll = a_lo * b_lo
    lh = a_lo * b_hi
    hl = a_hi * b_lo
    hh = a_hi * b_hi
    mid = (ll >> _S32) + (lh & _MASK32) + (hl & _MASK32)
    lo = (ll & _MASK32) | ((mid & _MASK32) << _S32)
    hi = hh + (lh >> _S32) + (hl >> _S32) + (mid >> _S32)
    return hi, lo


def philox4x64_10(counter, key):
    """Ten rounds of Philox4x64.

    counter: uint64 array [..., 4];  key: uint64 array [..., 2] (broadcast).
    Returns uint64 array [..., 4].
    """
    with np.errstate(over="ignore"):
        c = np.array(counter, dtype=np.uint64, copy=True)
        k = np.broadcast_to(np.asarray(key, dtype=np.uint64), c.shape[:-1] + (2,)).copy()
        x0, x1, x2, x3 = c[..., 0], c[..., 1], c[..., 2], c[..., 3]
        k0, k1 = k[..., 0], k[..., 1]
        for rnd in range(10):
            if rnd > 0:            # key schedule: Weyl sequence between rounds
                k0 = k0 + W0
                k1 = k1 + W1
            hi0, lo0 = _mulhilo(M0, x0)
            hi1, lo1 = _mulhilo(M1, x2)
            x0, x1, x2, x3 = hi1 ^ x1 ^ k0, lo1, hi0 ^ x3 ^ k1, lo0
        return np.stack([x0, x1, x2, x3], axis=-1)


def to_unit(r: np.ndarray) -> np.ndarray:
    """Map 64-bit words to doubles strictly inside (0, 1), exactly."""
    r = np.asarray(r, dtype=np.uint64)
    k = (r >> np.uint64(11)) | np.uint64(1)
    return k.astype(np.float64) * 2.0 ** -53


def vegas_uniforms(seed: int, iteration: int, subprocess: int, first_event: int,
                   n: int, ndim: int) -> np.ndarray:
    """Uniforms for events [first_event, first_event + n), SoA [ndim, n]."""
    ev = np.arange(first_event, first_event + n, dtype=np.uint64)
    out = np.empty((ndim, n), dtype=np.float64)
    nblk = (ndim + 3) // 4
    key = np.array([seed, 0], dtype=np.uint64)
    for b in range(nblk):
        ctr = np.zeros((n, 4), dtype=np.uint64)
        ctr[:, 0] = ev
        ctr[:, 1] = np.uint64(iteration)
        ctr[:, 2] = np.uint64(subprocess)
        ctr[:, 3] = np.uint64(b)
        words = philox4x64_10(ctr, key)
        for w in range(4):
            j = 4 * b + w
            if j < ndim:
                out[j] = to_unit(words[:, w])
    return out
