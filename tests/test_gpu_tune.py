"""The launch-shape tuner (mf_process_tune): whatever shape it keeps, the
integrand is the same bits as before tuning (the helicity sum is a fixed
pairwise tree for every number of lanes per event), and the shape is one of
the candidates."""
import numpy as np
import pytest

import workloads as W

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


@pytest.mark.parametrize("name,prec", [("gg_ttx", "fp64"), ("gg_ttxg", "mixed")])
def test_tuned_shape_gives_the_same_bits(env, name, prec):
    torch, api = env
    wl = W.WORKLOADS[name]
    proc = api.Process.from_workload(wl)
    x = torch.from_numpy(W.uniform_points(wl.ndim, 3001, 55)).cuda()
    before = proc.integrand(x, prec).cpu().numpy()
    block, ht = proc.tune(prec, n_sample=100_000)
    assert block in (128, 256) and ht in (8, 16, 32)
    after = proc.integrand(x, prec).cpu().numpy()
    assert np.array_equal(before, after)
    # a Vegas iteration after tuning: same bits as on an untuned twin
    twin = api.Process.from_workload(wl)
    ga, gb = api.Vegas(wl.ndim), api.Vegas(wl.ndim)
    ra = ga.iterate(proc, 50_000, 3, prec)
    rb = gb.iterate(twin, 50_000, 3, prec)
    assert ra == rb
    assert np.array_equal(ga.grid, gb.grid)
