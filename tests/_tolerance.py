"""Shared tolerance helpers of the GPU parity tests."""
import numpy as np

EPS = np.finfo(np.float64).eps


def relerr(got, ref):
    """|got - ref| / |ref|; 0 where both are zero, inf where only ref is."""
    got = np.asarray(got)
    ref = np.asarray(ref)
    both0 = (got == 0) & (ref == 0)
    out = np.full(got.shape, np.inf)
    nz = ref != 0
    out[nz] = np.abs(got[nz] - ref[nz]) / np.abs(ref[nz])
    out[both0] = 0.0
    return out


def fp64_tolerance(oracle, x):
    """1e-12 plus 64 eps x (the oracle's condition number of the point);
    where it is infinite (a density or the phase space vanishing) only the
    zero pattern is compared.  Returns (oracle f, tolerance)."""
    f, parts = oracle(x, return_parts=True)
    with np.errstate(invalid="ignore"):
        tol = 1e-12 + 64 * EPS * parts["condition"]
    # an undefined condition number goes with f = 0 (a density or the phase
    # space vanishing: only the zero pattern is compared); a point with a
    # value but no condition number gets the bare 1e-12
    tol = np.where(np.isnan(tol) & (f != 0), 1e-12, tol)
    return f, np.where(np.isnan(tol), np.inf, tol)
