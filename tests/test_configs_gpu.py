"""The workloads at their full sizes, in the launch configuration bench.py
times, checked against the CPU oracle (brute force, FP64 or exact integers):

* gauss64_1Mx128_knn10 (10^6 x 128 L2, k = 10): EVERY one of the 10,000
  queries, on the BF16 tensor-core path after the autotuner has chosen its
  launch parameters (as bench.py does) and on the plain FP32 path.
* dna_1M_r8 (10^6 DNA strings, radius 8): 256 of the 20,000 queries -- 224
  drawn at random and the 32 with the most answers -- on the 3-gram tiles and
  on the plain path.
* zipf2d_10M (10^7 2-D points, ~0.01% selectivity): six rounds of a
  10,000-query batch followed by 500 stream inserts and 500 stream deletes,
  with the 500,000-point batch update after the third round; per round 200
  queries (184 random, the 16 with the most answers) checked at the round's
  sequence number, on every path.
* wordvec_200000x300_cos_knn10 (2 * 10^5 x 300, angular distance, k = 10):
  1,024 of the 10,000 queries, drawn at random, with their FP64 keys, on the
  BF16 path after the shape and launch autotuners and on the plain FP32 path.
* multicol_200000_l2x128_cos300_knn10 (2 * 10^5 objects, an L2 column of
  128 and an angular column of 300 dimensions, distance = their sum): 256 of
  the 10,000 queries, kNN on both paths and a range query, FP64 sums exact.
* uniform_2Mx256_l1 (2 * 10^6 x 256 L1): 256 kNN queries (random and the
  largest k) and 256 range queries (random and the most answers) of the mixed
  batch; then the serving loop under 20,000 Poisson arrivals at 50,000/s and
  the 16 GB admission budget, with 256 served answers checked.

"Heaviest" queries are picked from the GPU's answer counts; only the choice
of which queries to check comes from the GPU, every expected value comes
from the oracle.
"""
import time

import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu
RTOL = 1e-5


@pytest.fixture(scope="module")
def env():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2404_00966_gb300 import build_ext
    build_ext.build()
    import paper_2404_00966_gb300 as g
    return g, torch


def _compare(got, idx, want, metric, label):
    """got: a Result over the whole batch (or a list of (ids, dist) per entry
    of idx); want: the oracle's CSR answers for the queries idx, in order."""
    off, ids, dist, _ = want
    bad = []
    for t, i in enumerate(idx):
        gi, gd = got[t][:2] if isinstance(got, list) else got.query(int(i))
        wi, wd = ids[off[t]:off[t + 1]], dist[off[t]:off[t + 1]]
        if not np.array_equal(gi, wi):
            bad.append((int(i), "ids", len(gi), len(wi)))
            continue
        if metric == "edit":
            ok = np.array_equal(gd, wd.astype(np.float32))
        else:
            ok = np.allclose(gd, wd, rtol=RTOL, atol=1e-30)
        if not ok:
            bad.append((int(i), "distances"))
    assert not bad, f"{label}: {len(bad)} of {len(idx)} queries differ from the oracle, first: {bad[:5]}"


def _heaviest(res, m):
    """The m queries of a batch with the most answers."""
    return np.argsort(-np.diff(np.asarray(res.offsets)), kind="stable")[:m]


def _pick(n, m_random, heavy, seed):
    """m_random queries drawn at random plus the given heavy ones, sorted."""
    rnd = np.random.default_rng(seed).choice(n, min(m_random, n), replace=False)
    return np.unique(np.concatenate([rnd, np.asarray(heavy, np.int64)]))


def test_gauss_full_size_every_query(env):
    g, torch = env
    wl = synth.gaussian_mixture()
    ix = g.Index.build(torch.from_numpy(wl.objects).cuda(), "l2", fanout=20, root_pivot=0)
    Qd = torch.from_numpy(wl.queries).cuda()
    every = np.arange(wl.nq)
    want = oracle.knn_query("l2", wl.objects, wl.queries, 10)
    ix.autotune(Qd, k=np.full(wl.nq, 10, np.int32), precision="bf16", reps=2)
    _compare(ix.knn(Qd, 10, precision="bf16"), every, want, "l2", "bf16 tiles, tuned")
    _compare(ix.knn(Qd, 10, precision="fp32"), every, want, "l2", "plain fp32")
    ix.close()


def test_wordvec_full_size(env):
    g, torch = env
    wl = synth.word_vectors()
    ix = g.Index.build(torch.from_numpy(wl.objects).cuda(), "cos", fanout=wl.fanout, root_pivot=0)
    Qd = torch.from_numpy(wl.queries).cuda()
    idx = _pick(wl.nq, 1024, [], seed=103)
    want = oracle.knn_query("cos", wl.objects, wl.queries[idx], 10)
    ix.autotune_shape(Qd[:2000], k=10, precision="bf16", candidates=4, reps=1)   # as bench.py does
    ix.autotune(Qd, k=wl.k, precision="bf16", reps=2)
    for prec in ("bf16", "fp32"):
        r = ix.knn(Qd, 10, precision=prec, keys=True)
        _compare(r, idx, want, "cos", f"wordvec {prec}")
        keys = np.concatenate([r.keys[r.offsets[i]:r.offsets[i + 1]] for i in idx])
        assert np.array_equal(keys, want[3]), f"wordvec {prec}: FP64 keys differ"
    ix.close()


def test_multicol_full_size(env):
    """The multi-column workload at full size (200,000 objects, an L2 column
    of 128 and an angular column of 300 dimensions), each column shaped as
    bench.py does: the whole 10,000-query batch runs, 256 sampled queries are
    compared with the oracle's brute force over the summed distance (kNN, and
    a range at 1.05 times the oracle's 10th sum)."""
    g, torch = env
    wl = synth.multi_columns()
    cols = [g.Index.build(torch.from_numpy(X).cuda(), m, fanout=wl.fanout, root_pivot=0)
            for X, m in zip(wl.objects, wl.metrics)]
    for ix, Q in zip(cols, wl.queries):
        ix.autotune_shape(torch.from_numpy(Q[:2000]).cuda(), k=10, precision="bf16", candidates=4, reps=1)
    idx = _pick(wl.queries[0].shape[0], 256, [], seed=104)
    qs = [Q[idx] for Q in wl.queries]
    want = oracle.multi_knn(wl.metrics, wl.objects, qs, 10)
    for prec in ("bf16", "fp32"):
        r = g.multi_knn(cols, wl.queries, wl.k, precision=prec)
        assert np.array_equal(np.diff(r.offsets), np.full(wl.queries[0].shape[0], 10))
        ids = np.concatenate([r.ids[r.offsets[i]:r.offsets[i + 1]] for i in idx])
        sums = np.concatenate([r.keys[r.offsets[i]:r.offsets[i + 1]] for i in idx])
        assert np.array_equal(ids, want[1]), f"multicol {prec}: ids differ"
        assert np.array_equal(sums, want[2]), f"multicol {prec}: FP64 sums differ"
    radii = (1.05 * want[2][9::10]).astype(np.float32)
    want_r = oracle.multi_range(wl.metrics, wl.objects, qs, radii)
    r = g.multi_range(cols, qs, radii, precision="bf16")
    assert np.array_equal(r.offsets, want_r[0]) and np.array_equal(r.ids, want_r[1])
    assert np.array_equal(r.keys, want_r[2])
    for ix in cols:
        ix.close()


def test_dna_full_size(env):
    g, torch = env
    wl = synth.dna_like()
    objs = (torch.from_numpy(wl.objects.data).cuda(), torch.from_numpy(wl.objects.offsets).cuda())
    ix = g.Index.build(objs, "edit", fanout=wl.fanout, root_pivot=0)
    qd = (torch.from_numpy(wl.queries.data).cuda(), torch.from_numpy(wl.queries.offsets).cuda())
    rd = torch.from_numpy(wl.radii).cuda()
    res = {prec: ix.range(qd, rd, precision=prec) for prec in ("bf16", "fp32")}   # 3-gram tiles, plain path
    idx = _pick(wl.nq, 224, _heaviest(res["bf16"], 32), seed=102)
    assert idx.shape[0] >= 256
    want = oracle.range_query("edit", wl.objects, wl.queries.take(idx), wl.radii[idx])
    for prec, r in res.items():
        _compare(r, idx, want, "edit", f"dna {prec}")
    ix.close()


class _Visibility:
    """Host model of the sequence numbers of stream updates (Section 4.4):
    object o is visible to a query at sequence s iff ins[o] < s < del[o]."""

    def __init__(self, X, seq0):
        self.P = [X]
        self.ins = [np.full(X.shape[0], -1, np.int64)]
        self.dele = [np.full(X.shape[0], np.iinfo(np.int64).max, np.int64)]
        self.live = np.ones(X.shape[0], bool)
        self.seq = seq0

    def insert(self, pts):
        self.P.append(pts)
        self.ins.append(self.seq + np.arange(pts.shape[0], dtype=np.int64))
        self.dele.append(np.full(pts.shape[0], np.iinfo(np.int64).max, np.int64))
        self.live = np.concatenate([self.live, np.ones(pts.shape[0], bool)])
        self.seq += pts.shape[0]

    def delete(self, ids):
        dele = np.concatenate(self.dele)
        dele[ids] = self.seq + np.arange(ids.shape[0], dtype=np.int64)
        self.dele = [dele]
        self.live[ids] = False
        self.seq += ids.shape[0]

    def arrays(self):
        return np.concatenate(self.P), np.concatenate(self.ins), np.concatenate(self.dele)


def test_zipf2d_full_size_with_update_rounds(env):
    g, torch = env
    wl = synth.zipf_clusters_2d(nq=60_000)
    ix = g.Index.build(torch.from_numpy(wl.objects).cuda(), "l2", fanout=20, root_pivot=0, cache_limit=4096)
    vis = _Visibility(wl.objects, ix.info()["seq"])
    upd = synth.zipf_points(wl.extra["centers"], wl.extra["weights"], 0.01, 3_000, seed=2)
    bulk = synth.zipf_points(wl.extra["centers"], wl.extra["weights"], 0.01, 500_000, seed=5)
    drng = np.random.default_rng(3)
    r = np.float32(0.0025)   # about a thousand answers per query on this mixture
    nb = 10_000
    radii = torch.full((nb,), float(r), dtype=torch.float32, device="cuda")
    checked = 0
    for rnd in range(6):
        qb = wl.queries[rnd * nb:(rnd + 1) * nb]
        Qd = torch.from_numpy(qb).cuda()
        res = {prec: ix.range(Qd, radii, precision=prec) for prec in ("bf16", "fp32")}
        idx = _pick(nb, 184, _heaviest(res["bf16"], 16), seed=200 + rnd)
        P, ins, dele = vis.arrays()
        assert ix.info()["seq"] == vis.seq
        want = oracle.range_query("l2", P, qb[idx], np.full(idx.shape[0], r, np.float32), ins, dele,
                                  np.full(idx.shape[0], vis.seq, np.int64))
        for prec, got in res.items():
            _compare(got, idx, want, "l2", f"zipf2d round {rnd} {prec}")
        checked += idx.shape[0]
        # 10% updates between query batches: 500 inserts, then 500 deletes of live objects
        ix.insert(upd[rnd * 500:(rnd + 1) * 500])
        vis.insert(upd[rnd * 500:(rnd + 1) * 500])
        victims = drng.choice(np.nonzero(vis.live)[0], 500, replace=False).astype(np.int64)
        assert ix.delete(victims) == 0
        vis.delete(victims)
        if rnd == 2:
            ix.batch_update(bulk)   # rebuild with 500,000 more points (Section 4.4)
            vis.insert(bulk)
    assert checked >= 1200
    ix.close()


def test_uniform_l1_full_size_mixed_and_served(env):
    g, torch = env
    nreq = 20_000
    wl = synth.uniform_cube(n=2_000_000, dim=256, nq=nreq)
    ix = g.Index.build(torch.from_numpy(wl.objects).cuda(), "l1", fanout=20, root_pivot=0)
    Qd = torch.from_numpy(wl.queries[:4000]).cuda()
    is_knn, ks = synth.mixed_requests(nreq, seed=1)
    cal = ix.knn(Qd[:200], 100)
    r = np.float32(np.mean([cal.query(i)[1][-1] for i in range(200)]))   # about 100 answers
    kq = ks[:4000].copy()
    radii = np.full(4000, r, np.float32)
    res_k = {p: ix.knn(Qd, torch.from_numpy(kq).cuda(), precision=p) for p in ("bf16", "fp32")}
    res_r = {p: ix.range(Qd, torch.from_numpy(radii).cuda(), precision=p) for p in ("bf16", "fp32")}
    idx_k = _pick(4000, 240, np.argsort(-kq, kind="stable")[:16], seed=105)
    idx_r = _pick(4000, 240, _heaviest(res_r["bf16"], 16), seed=106)
    want_k = oracle.knn_query("l1", wl.objects, wl.queries[idx_k], kq[idx_k])
    want_r = oracle.range_query("l1", wl.objects, wl.queries[idx_r], radii[idx_r])
    for p in ("bf16", "fp32"):        # node-major FP32 tiles, then the plain path
        _compare(res_k[p], idx_k, want_k, "l1", f"l1 knn {p}")
        _compare(res_r[p], idx_r, want_r, "l1", f"l1 range {p}")
    # served: open-loop Poisson arrivals through the continuous-batching loop
    arrivals = synth.poisson_arrivals(nreq, 50_000.0, seed=1)
    sv = g.Server(ix, max_batch=1024, n_streams=2, precision="bf16", result_budget=16 << 30,
                  batch_quantum=64)   # as bench.py serves
    tickets = []
    start = time.perf_counter()
    for i in range(nreq):
        while time.perf_counter() - start < arrivals[i]:
            pass
        tickets.append(sv.submit(wl.queries[i], "knn" if is_knn[i] else "range", int(ks[i]) if is_knn[i] else r))
    served = [sv.wait(t) for t in tickets]
    st = sv.stats()
    sv.stop()
    assert st["requests"] == nreq and st["max_in_flight"] <= 16 << 30
    knn_ids, rng_ids = np.nonzero(is_knn)[0], np.nonzero(~is_knn)[0]
    heavy_k = knn_ids[np.argsort(-ks[knn_ids], kind="stable")[:16]]
    heavy_r = rng_ids[np.argsort(-np.array([len(served[i][0]) for i in rng_ids]), kind="stable")[:16]]
    pick = _pick(nreq, 224, np.concatenate([heavy_k, heavy_r]), seed=107)
    pk, pr = pick[is_knn[pick]], pick[~is_knn[pick]]
    _compare([served[i] for i in pk], pk, oracle.knn_query("l1", wl.objects, wl.queries[pk], ks[pk]), "l1",
             "served knn")
    _compare([served[i] for i in pr], pr,
             oracle.range_query("l1", wl.objects, wl.queries[pr], np.full(pr.shape[0], r, np.float32)), "l1",
             "served range")
    ix.close()
