"""The launch-shape tuner (mf_process_tune): the shape it keeps is one of
the candidates; block size and lanes per point never change the bits (the
helicity sum is a fixed pairwise tree for every number of lanes per event);
a compiled-in minimum of resident blocks may change the last bits only."""
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
    info = proc.kernel_info(prec)
    after = proc.integrand(x, prec).cpu().numpy()
    assert np.array_equal(before == 0, after == 0)
    if info["min_blocks"] == 0:
        assert np.array_equal(before, after)
    else:
        nz = before != 0
        assert np.max(np.abs(after[nz] / before[nz] - 1)) < (1e-12 if prec == "fp64" else 1e-5)
    # an untuned twin with the same block and lanes gives the same bits
    twin = api.Process.from_workload(wl, options={"block": block, "lanes": ht, "min_blocks": info["min_blocks"]})
    twin_f = twin.integrand(x, prec).cpu().numpy()
    assert np.array_equal(after, twin_f)
