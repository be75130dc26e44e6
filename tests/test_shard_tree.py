"""The pairwise tree over Vegas chunks that makes a data-parallel iteration
bit-identical to the single-device one (host only, no GPU).

* the tree's value is checked against its recursive definition, written out
  here independently, and against exact sums (integers);
* the frontiers of any split of the chunk range partition it, and combining
  the per-rank frontier values reproduces the single-range root bit for bit;
* malformed node sets (missing, duplicate, overlapping, out of range) are
  rejected with MF_EINVAL;
* two gloo ranks exchange their nodes as the data-parallel benchmark does
  (fixed-size records, one all-gather) and both rebuild the same root as one
  rank alone.
"""
import socket

import numpy as np
import pytest


@pytest.fixture(scope="module")
def api():
    import __graft_entry__ as g
    g.build()
    from paper_2106_10279_gb300 import api
    return api


def _definition(leaves, level, index):
    """Node (level, index) straight from the definition: the sum of its two
    children, or the left child alone when the right one has no chunk."""
    n = leaves.shape[0]
    if level == 0:
        return leaves[index].copy()
    left = _definition(leaves, level - 1, 2 * index)
    if ((2 * index + 1) << (level - 1)) < n:
        return left + _definition(leaves, level - 1, 2 * index + 1)
    return left


def _leaf_records(leaves, c0, c1):
    K = leaves.shape[1]
    rec = np.zeros((c1 - c0, 2 + K))
    rec[:, 0] = 0
    rec[:, 1] = np.arange(c0, c1)
    rec[:, 2:] = leaves[c0:c1]
    return rec


def _rank_nodes(api, leaves, c0, c1):
    n = leaves.shape[0]
    ids = api.mf_tree_frontier(c0, c1, n)
    K = leaves.shape[1]
    out = np.zeros((len(ids), 2 + K))
    for j, (l, i) in enumerate(ids):
        lo, hi = int(i) << int(l), min((int(i) + 1) << int(l), n)
        out[j, :2] = (l, i)
        out[j, 2:] = api.mf_tree_reduce(_leaf_records(leaves, lo, hi), n, int(l), int(i))
    return out


@pytest.mark.parametrize("n", [1, 2, 3, 7, 8, 9, 100, 257, 1000])
def test_root_matches_definition(api, n):
    rng = np.random.default_rng(n)
    leaves = rng.standard_normal((n, 3)) * np.exp(rng.uniform(-30, 30, (n, 3)))
    L = api.tree_levels(n)
    root = api.mf_tree_reduce(_leaf_records(leaves, 0, n), n, L, 0)
    assert np.array_equal(root, _definition(leaves, L, 0))
    # integers below 2^53: every order gives the exact sum
    ints = rng.integers(0, 2 ** 40, (n, 2)).astype(np.float64)
    r = api.mf_tree_reduce(_leaf_records(ints, 0, n), n, L, 0)
    assert np.array_equal(r, ints.sum(axis=0))


@pytest.mark.parametrize("n", [1, 5, 16, 17, 1000, 9766])
def test_frontiers_partition_every_split(api, n):
    rng = np.random.default_rng(100 + n)
    for _ in range(20):
        R = int(rng.integers(1, 6))
        cuts = np.sort(rng.integers(0, n + 1, R - 1))
        bounds = [0, *cuts.tolist(), n]
        covered = np.zeros(n, dtype=int)
        for c0, c1 in zip(bounds[:-1], bounds[1:]):
            for l, i in api.mf_tree_frontier(c0, c1, n):
                lo, hi = int(i) << int(l), min((int(i) + 1) << int(l), n)
                assert c0 <= lo and (hi <= c1)
                covered[lo:hi] += 1
        assert np.all(covered == 1)
        # a frontier is short: at most two nodes per level
        assert len(api.mf_tree_frontier(0, n, n)) == 1
        assert all(len(api.mf_tree_frontier(a, b, n)) <= 2 * api.tree_levels(n) + 2
                   for a, b in zip(bounds[:-1], bounds[1:]))


@pytest.mark.parametrize("n", [3, 64, 65, 1000, 9766])
def test_sharded_root_is_bit_identical(api, n):
    rng = np.random.default_rng(200 + n)
    leaves = rng.standard_normal((n, 5)) * np.exp(rng.uniform(-20, 20, (n, 5)))
    L = api.tree_levels(n)
    ref = api.mf_tree_reduce(_leaf_records(leaves, 0, n), n, L, 0)
    for R in (1, 2, 3, 4, 7):
        bounds = [n * r // R for r in range(R + 1)]
        nodes = np.concatenate([_rank_nodes(api, leaves, a, b) for a, b in zip(bounds[:-1], bounds[1:])])
        perm = rng.permutation(nodes.shape[0])               # arrival order does not matter
        got = api.mf_tree_reduce(nodes[perm], n, L, 0)
        assert np.array_equal(got, ref), R
    # a plain left-to-right sum over the chunks rounds differently: the fixed
    # tree, not luck, makes the shards agree
    if n >= 64:
        seq = np.zeros(leaves.shape[1])
        for row in leaves:
            seq = seq + row
        assert not np.array_equal(seq, ref)


def test_malformed_node_sets_are_rejected(api):
    from paper_2106_10279_gb300 import _lib as L
    n = 10
    leaves = np.arange(n * 2, dtype=np.float64).reshape(n, 2)
    rec = _leaf_records(leaves, 0, n)
    Lv = api.tree_levels(n)
    for bad in (rec[1:],                                  # missing chunk 0
                np.concatenate([rec, rec[:1]]),           # duplicate
                np.concatenate([rec, np.array([[1, 0, 0.0, 0.0]])]),   # overlaps chunks 0, 1
                np.concatenate([rec, np.array([[0, 10, 0.0, 0.0]])]),  # beyond the last chunk
                np.concatenate([rec, np.array([[0.5, 3, 0.0, 0.0]])])):  # not an integer level
        with pytest.raises(L.MfError) as e:
            api.mf_tree_reduce(bad, n, Lv, 0)
        assert e.value.status == L.MF_EINVAL
    with pytest.raises(L.MfError):
        api.mf_tree_frontier(3, 2, n)
    with pytest.raises(L.MfError):
        api.mf_tree_frontier(0, n + 1, n)
    with pytest.raises(L.MfError):
        api.mf_tree_reduce(rec, n, Lv, 1)            # node beyond the last chunk
    # a node above the root covers the same chunks and has the root's value
    assert np.array_equal(api.mf_tree_reduce(rec, n, Lv + 1, 0), api.mf_tree_reduce(rec, n, Lv, 0))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _gloo_rank(rank, world, port, n, q):
    import torch.distributed as dist
    import __graft_entry__ as g
    g.build()
    from paper_2106_10279_gb300 import api
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=world)
    try:
        rng = np.random.default_rng(7)
        leaves = rng.standard_normal((n, 4)) * np.exp(rng.uniform(-25, 25, (n, 4)))
        nchunks = n
        c0, c1 = nchunks * rank // world, nchunks * (rank + 1) // world
        mine = _rank_nodes(api, leaves, c0, c1)
        # the exchange of the data-parallel benchmark: fixed-size records,
        # one all-gather
        import torch
        K = leaves.shape[1]
        buf = torch.from_numpy(api.pack_nodes(mine, K))
        parts = [torch.empty_like(buf) for _ in range(world)]
        dist.all_gather(parts, buf)
        allnodes = api.unpack_nodes(torch.stack(parts).numpy(), K)
        got = api.mf_tree_reduce(allnodes, n, api.tree_levels(n), 0)
        ref = api.mf_tree_reduce(_leaf_records(leaves, 0, n), n, api.tree_levels(n), 0)
        q.put((rank, bool(np.array_equal(got, ref)), got.tobytes()))
    except Exception as e:                        # report instead of leaving the parent waiting
        q.put((rank, False, repr(e).encode()))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_rebuild_the_same_root(api):
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    n = 9766                                  # chunks of a 4e7-point iteration
    procs = [ctx.Process(target=_gloo_rank, args=(r, 2, port, n, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = [q.get(timeout=240) for _ in procs]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert all(ok for _, ok, _ in res), res
    assert res[0][2] == res[1][2]
