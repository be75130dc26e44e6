"""The compile-time self-check of the helicity-pair program.

gg -> tt~g generated with amplitude units (the default) and the searched
amplitude order: its FP64 pair program, built by the device assembler at
its default optimisation level, was wrong at every point while the same
source at levels 0 and 1, the host build and every other program form were
right.  The create-time check compares the pair program with the
single-helicity program of the same kernel and rebuilds the kernel at a
lower level when they disagree; the process then matches the oracle and a
process without units.
"""
import numpy as np
import pytest

import workloads as W
from _tolerance import fp64_tolerance, relerr

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__ as g
    g.build()
    from paper_2106_10279_gb300 import api
    return torch, api


@pytest.mark.parametrize("options", [{"amplitude_units": 1}, {"amplitude_units": 1, "order_search": 1000},
                                     {"amplitude_units": 1, "ptxas_level": 2}])
def test_units_in_short_programs_give_correct_values(env, oracle_processes, options):
    torch, api = env
    from oracle.integrand import Integrand
    wl = W.GG_TTXG
    x = W.uniform_points(wl.ndim, 600, 71)
    xd = torch.from_numpy(x).cuda()
    p = api.Process.from_workload(wl, options=options)
    default = api.Process.from_workload(wl, options={"amplitude_units": 0})
    f64 = p.integrand(xd, "fp64").cpu().numpy()
    ref, tol = fp64_tolerance(Integrand(wl, process=oracle_processes("gg_ttxg")), x)
    assert np.array_equal(f64 == 0, ref == 0)
    assert np.all(relerr(f64, ref) <= tol)
    fd = default.integrand(xd, "fp64").cpu().numpy()
    nz = fd != 0
    assert np.max(np.abs(f64[nz] / fd[nz] - 1)) < 1e-12
    fm = p.integrand(xd, "mixed").cpu().numpy()
    r = relerr(fm, ref)[ref != 0]
    assert np.median(r) <= 1e-5 and r.max() <= 1e-3
