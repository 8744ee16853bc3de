"""Sharded answers and index files, host side (CPU only, no device):

* gts_merge_knn / gts_merge_range turn the answers of shards over disjoint
  object sets into the answers of one index over their union.  The shards'
  answers here are the oracle's own over each slice, so the merge is checked
  against the oracle over all objects, with exact ties across shards (integer
  points) decided by global id.
* The same merge after an exchange between two gloo ranks, each holding one
  shard (the exchange a sharded deployment would make).
* gts_load rejects a file that is not an index, or a truncated one, before it
  touches a device.
"""
import os
import socket

import numpy as np
import pytest

import oracle

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


@pytest.fixture(scope="module")
def g():
    from paper_2404_00966_gb300 import build_ext
    build_ext.build()
    import paper_2404_00966_gb300 as gts
    return gts


def _points(n, nq, seed):
    rng = np.random.default_rng(seed)
    X = rng.integers(0, 4, size=(n, 3)).astype(np.float32)      # many exactly tied distances
    Q = rng.integers(0, 4, size=(nq, 3)).astype(np.float32)
    return X, Q


def _shard_answers(metric, X, Q, cuts, k=None, radii=None):
    parts = []
    for s in range(len(cuts) - 1):
        sl = X[cuts[s]:cuts[s + 1]]
        if k is not None:
            parts.append(oracle.knn_query(metric, sl, Q, k))          # (offsets, ids, dist, keys)
        else:
            off, ids, dist, _ = oracle.range_query(metric, sl, Q, radii)
            parts.append((off, ids, dist))
    return parts


@pytest.mark.parametrize("metric", ["l2", "l1"])
def test_merge_matches_the_union(g, metric):
    X, Q = _points(3000, 40, seed=7)
    cuts = [0, 700, 701, 1900, 3000]                               # a one-object shard too
    ks = np.random.default_rng(8).integers(1, 60, size=40).astype(np.int32)
    parts = _shard_answers(metric, X, Q, cuts, k=ks)
    off, ids, dist, keys = g.merge_knn(parts, cuts[:-1], ks)
    w_off, w_ids, w_dist, w_keys = oracle.knn_query(metric, X, Q, ks)
    assert np.array_equal(off, w_off) and np.array_equal(ids, w_ids) and np.array_equal(keys, w_keys)
    assert np.allclose(dist, w_dist, rtol=1e-6)
    radii = np.full(40, 1.5, np.float32)
    parts = _shard_answers(metric, X, Q, cuts, radii=radii)
    off, ids, dist, _ = g.merge_range(parts, cuts[:-1])
    w_off, w_ids, w_dist, _ = oracle.range_query(metric, X, Q, radii)
    assert np.array_equal(off, w_off) and np.array_equal(ids, w_ids)
    assert np.allclose(dist, w_dist, rtol=1e-6)


def test_merge_rejects_parts_without_keys(g):
    X, Q = _points(100, 3, seed=9)
    parts = [(p[0], p[1], p[2]) for p in _shard_answers("l2", X, Q, [0, 50, 100], k=4)]
    with pytest.raises(g.GTSError):
        g.merge_knn(parts, [0, 50], 4)


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import paper_2404_00966_gb300 as gts
    X, Q = _points(2000, 25, seed=11)
    cuts = [0, 1200, 2000]
    mine = oracle.knn_query("l2", X[cuts[rank]:cuts[rank + 1]], Q, 9)   # this rank's shard
    gathered = [None] * world
    dist.all_gather_object(gathered, [np.asarray(a) for a in mine])
    off, ids, _, keys = gts.merge_knn(gathered, cuts[:-1], 9)
    w_off, w_ids, _, w_keys = oracle.knn_query("l2", X, Q, 9)
    out[rank] = bool(np.array_equal(off, w_off) and np.array_equal(ids, w_ids) and np.array_equal(keys, w_keys))
    dist.barrier()
    dist.destroy_process_group()


def test_sharded_knn_merge_across_gloo_ranks(g):
    port = _free_port()
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_rank, args=(2, port, out), nprocs=2, join=True)
        assert dict(out) == {0: True, 1: True}


def test_load_rejects_bad_files(g, tmp_path):
    bad = tmp_path / "bad.gts"
    bad.write_bytes(b"not an index at all")
    with pytest.raises(g.GTSError) as e:
        g.Index.load(str(bad))
    assert e.value.status == 1
    trunc = tmp_path / "trunc.gts"
    trunc.write_bytes(b"GTSIDX01" + (1).to_bytes(4, "little") + b"\x02\x00")
    with pytest.raises(g.GTSError) as e:
        g.Index.load(str(trunc))
    assert e.value.status == 1
    with pytest.raises(g.GTSError):
        g.Index.load(str(tmp_path / "missing.gts"))
