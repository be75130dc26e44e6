"""Data-parallel Vegas iterations and checkpoints on the device.

* an iteration split into shards (2, 3 and 5 ranks, uneven, one empty) and
  recombined with mf_vegas_shard_finish gives the same bits as
  mf_vegas_iterate: estimate, error, histogram, counts and refined grid, over
  two iterations in a row;
* a grid saved after two iterations and loaded into a fresh grid continues
  with the same bits as the uninterrupted run; malformed checkpoints are
  rejected.
"""
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
    return api


def _state(v):
    h, c = v.histogram()
    return v.grid.copy(), h.copy(), c.copy()


def _same(a, b):
    keys = ("iteration", "n_events", "n_nonzero", "n_nan", "integral", "error", "sigma", "sigma_error", "chi2_dof")
    return all(a[k] == b[k] for k in keys)


@pytest.mark.parametrize("name,n,prec", [("gg_ttx", 100_003, "fp64"), ("gg_ttxg", 50_000, "mixed")])
def test_shards_are_bit_identical_to_one_iteration(env, name, n, prec):
    api = env
    wl = W.WORKLOADS[name]
    proc = api.Process.from_workload(wl)
    ref = api.Vegas(wl.ndim)
    seed = 11
    nchunks = (n + 4095) // 4096
    splits = {2: [0, nchunks // 2, nchunks],
              3: [0, 1, nchunks - 3, nchunks],
              5: [0, 4, 4, 9, nchunks - 1, nchunks]}      # includes an empty shard
    grids = {R: api.Vegas(wl.ndim) for R in splits}
    for it in range(2):
        r_ref = ref.iterate(proc, n, seed, prec)
        s_ref = _state(ref)
        for R, b in splits.items():
            v = grids[R]
            nodes = [v.iterate_shard(proc, n, b[r], b[r + 1], seed, subprocess=0, precision=prec)
                     for r in range(R)]
            if R == 5:
                assert nodes[1].shape[0] == 0                # chunks [4, 4)
            r = v.finish_shards(n, np.concatenate(nodes))
            assert _same(r, r_ref), (R, it, r, r_ref)
            for x, y in zip(_state(v), s_ref):
                assert np.array_equal(x, y), (R, it)


def test_shard_finish_rejects_incomplete_nodes(env):
    api = env
    from paper_2106_10279_gb300 import _lib as L
    wl = W.GG_TTX
    proc = api.Process.from_workload(wl)
    v = api.Vegas(wl.ndim)
    n = 20_000
    nodes = v.iterate_shard(proc, n, 0, 2, 3)
    with pytest.raises(L.MfError) as e:
        v.finish_shards(n, nodes)              # chunks 2..4 missing
    assert e.value.status == L.MF_EINVAL
    shape_before = api.mf_vegas_get_grid(v.handle)
    assert np.array_equal(shape_before, api.Vegas(wl.ndim).grid)   # nothing refined


def test_checkpoint_resumes_bit_identically(env):
    api = env
    from paper_2106_10279_gb300 import _lib as L
    wl = W.GG_TTX
    proc = api.Process.from_workload(wl)
    a = api.Vegas(wl.ndim)
    n = 60_000
    for _ in range(2):
        a.iterate(proc, n, 5)
    blob = a.save()
    b = api.Vegas(wl.ndim)
    b.load(blob)
    assert b.save() == blob
    for _ in range(2):
        ra = a.iterate(proc, n, 5)
        rb = b.iterate(proc, n, 5)
        assert _same(ra, rb)
        for x, y in zip(_state(a), _state(b)):
            assert np.array_equal(x, y)
    # wrong shape, truncated, corrupted tag, non-monotone edges
    with pytest.raises(L.MfError):
        api.Vegas(wl.ndim + 1).load(blob)
    with pytest.raises(L.MfError):
        api.Vegas(wl.ndim).load(blob[:-8])
    with pytest.raises(L.MfError):
        api.Vegas(wl.ndim).load(b"X" + blob[1:])
    bad = bytearray(blob)
    off = 32 + 8 * 3                                      # header, then edge 3 of dimension 0
    bad[off:off + 8] = np.float64(2.0).tobytes()
    with pytest.raises(L.MfError):
        api.Vegas(wl.ndim).load(bytes(bad))
