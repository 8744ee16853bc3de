"""The workloads at their full sizes, in the launch configuration bench.py
times: the GPU answers every query of the batch; the CPU oracle checks a
seeded sample of the answers one by one.

* gauss64_1Mx128_knn10: 10^6 x 128 L2, 10,000 kNN queries (k = 10), BF16
  tiles and the plain FP32 path.
* dna_1M_r8: 10^6 DNA strings, 20,000 range queries of radius 8.
* zipf2d_10M: 10^7 2-D points, range queries at ~0.01% selectivity, after
  stream inserts / deletes and a batch update (sequence-number visibility).
* uniform_2Mx256_l1: 2 * 10^6 x 256 L1, mixed range and kNN (k up to 100).
"""
import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu
RTOL = 1e-5
SAMPLE = 24


@pytest.fixture(scope="module")
def env():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2404_00966_gb300 import build_ext
    build_ext.build()
    import paper_2404_00966_gb300 as g
    return g, torch


def _check(res, idx, want, metric):
    off, ids, dist, _ = want
    for t, i in enumerate(idx):
        gi, gd = res.query(int(i))
        wi, wd = ids[off[t]:off[t + 1]], dist[off[t]:off[t + 1]]
        assert np.array_equal(gi, wi), f"query {i}: ids differ"
        if metric == "edit":
            assert np.array_equal(gd, wd.astype(np.float32)), f"query {i}: distances differ"
        else:
            assert np.allclose(gd, wd, rtol=RTOL, atol=1e-30), f"query {i}: distances differ"


def test_gauss_full_size(env):
    g, torch = env
    wl = synth.gaussian_mixture()
    ix = g.Index.build(torch.from_numpy(wl.objects).cuda(), "l2", fanout=20, root_pivot=0)
    Qd = torch.from_numpy(wl.queries).cuda()
    idx = np.random.default_rng(101).choice(wl.nq, SAMPLE, replace=False)
    want = oracle.knn_query("l2", wl.objects, wl.queries[idx], 10)
    for prec in ("bf16", "fp32"):
        _check(ix.knn(Qd, 10, precision=prec), idx, want, "l2")
    ix.close()


def test_dna_full_size(env):
    g, torch = env
    wl = synth.dna_like()
    objs = (torch.from_numpy(wl.objects.data).cuda(), torch.from_numpy(wl.objects.offsets).cuda())
    ix = g.Index.build(objs, "edit", fanout=wl.fanout, root_pivot=0)
    idx = np.random.default_rng(102).choice(wl.nq, 12, replace=False)
    want = oracle.range_query("edit", wl.objects, wl.queries.take(idx), wl.radii[idx])
    for prec in ("bf16", "fp32"):   # the 3-gram tiles, then the plain path
        res = ix.range((torch.from_numpy(wl.queries.data).cuda(), torch.from_numpy(wl.queries.offsets).cuda()),
                       torch.from_numpy(wl.radii).cuda(), precision=prec)
        _check(res, idx, want, "edit")
    ix.close()


def test_zipf2d_full_size_with_updates(env):
    g, torch = env
    wl = synth.zipf_clusters_2d(nq=20_000)
    X = wl.objects
    ix = g.Index.build(torch.from_numpy(X).cuda(), "l2", fanout=20, root_pivot=0, cache_limit=4096)
    s0 = ix.info()["seq"]
    ins = synth.zipf_points(wl.extra["centers"], wl.extra["weights"], 0.01, 3000, seed=2)
    ix.insert(ins)                                        # stays in the cache list
    dele = np.random.default_rng(3).choice(X.shape[0] + 3000, 3000, replace=False)
    missing = ix.delete(dele)
    assert missing == 0
    s1 = ix.info()["seq"]
    P = np.concatenate([X, ins])
    ins_seq = np.concatenate([np.full(X.shape[0], -1), s0 + np.arange(3000)]).astype(np.int64)
    del_seq = np.full(P.shape[0], np.iinfo(np.int64).max, np.int64)
    del_seq[dele] = s0 + 3000 + np.arange(3000)
    r = np.float32(0.0025)   # about a thousand results per query on this mixture
    radii = np.full(wl.nq, r, np.float32)
    idx = np.random.default_rng(104).choice(wl.nq, SAMPLE, replace=False)
    qs = np.full(SAMPLE, s1, np.int64)
    want = oracle.range_query("l2", P, wl.queries[idx], radii[idx], ins_seq, del_seq, qs)
    for prec in ("fp32", "bf16"):
        res = ix.range(torch.from_numpy(wl.queries).cuda(), torch.from_numpy(radii).cuda(), precision=prec)
        _check(res, idx, want, "l2")
    # batch update (rebuild) with 500,000 more points
    bulk = synth.zipf_points(wl.extra["centers"], wl.extra["weights"], 0.01, 500_000, seed=5)
    ix.batch_update(bulk)
    s2 = ix.info()["seq"]
    P2 = np.concatenate([P, bulk])
    ins2 = np.concatenate([ins_seq, s1 + np.arange(500_000)]).astype(np.int64)
    del2 = np.concatenate([del_seq, np.full(500_000, np.iinfo(np.int64).max, np.int64)])
    want = oracle.range_query("l2", P2, wl.queries[idx], radii[idx], ins2, del2, np.full(SAMPLE, s2, np.int64))
    res = ix.range(torch.from_numpy(wl.queries).cuda(), torch.from_numpy(radii).cuda())
    _check(res, idx, want, "l2")
    ix.close()


def test_uniform_l1_full_size_mixed(env):
    g, torch = env
    wl = synth.uniform_cube(n=2_000_000, dim=256, nq=4000)
    ix = g.Index.build(torch.from_numpy(wl.objects).cuda(), "l1", fanout=20, root_pivot=0)
    Qd = torch.from_numpy(wl.queries).cuda()
    is_knn, ks = synth.mixed_requests(wl.nq, seed=1)
    idx = np.random.default_rng(105).choice(wl.nq, 16, replace=False)
    kq = ks.copy()
    want_k = oracle.knn_query("l1", wl.objects, wl.queries[idx], kq[idx])
    cal = ix.knn(Qd[:200], 100)
    r = np.float32(np.mean([cal.query(i)[1][-1] for i in range(200)]))
    radii = np.full(wl.nq, r, np.float32)
    want_r = oracle.range_query("l1", wl.objects, wl.queries[idx], radii[idx])
    for prec in ("bf16", "fp32"):        # node-major FP32 tiles, then the plain path
        _check(ix.knn(Qd, torch.from_numpy(kq).cuda(), precision=prec), idx, want_k, "l1")
        _check(ix.range(Qd, torch.from_numpy(radii).cuda(), precision=prec), idx, want_r, "l1")
    ix.close()
