"""Parity of the angular (cosine) distance with the CPU oracle, through the C
ABI: the distance between two word vectors is the angle between them, Table
2's cosine distance read as a metric.  The index is an L2 tree over the unit
vectors; every reported answer takes its FP64 key 1 - cos on the raw vectors
in the oracle's operation order, so ids and keys match the oracle exactly and
angles within 1e-5 relative.

Inputs: direction clusters with exact scalar multiples of other rows (key 0
up to rounding), antipodal rows (angle pi) and exact duplicates; dimensions
3 (the table scan), 24 and 300 (the Vector data's width, tensor-core tiles).
"""
import numpy as np
import pytest

import oracle
from synth import small_vectors

pytestmark = pytest.mark.gpu
RTOL = 1e-5


@pytest.fixture(scope="module")
def gts():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2404_00966_gb300 import build_ext
    build_ext.build()
    import paper_2404_00966_gb300 as g
    return g


def cos_case(n, dim, nq, seed):
    X, Q = small_vectors(n, dim, nq, seed, kind="gauss", dup_frac=0.05)
    rng = np.random.default_rng(seed + 1000)
    m = n // 20
    src = rng.integers(0, n, size=m)
    dst = rng.choice(n, size=2 * m, replace=False)
    X[dst[:m]] = X[src] * rng.choice(np.float32([0.5, 2.0, 4.0, 0.25]), size=(m, 1))   # same direction
    X[dst[m:]] = -X[src]                                                                   # antipodal
    Q[: nq // 4] = X[rng.integers(0, n, size=nq // 4)] * np.float32(3.0)                  # queries on a row's ray
    return X, Q


def angle_radii(X, Q, frac, seed):
    rng = np.random.default_rng(seed)
    sample = X[rng.choice(X.shape[0], size=min(400, X.shape[0]), replace=False)]
    return np.array([np.quantile(oracle.distances_to("cos", sample, q), frac) for q in Q], np.float32)


def assert_same(res, want, label):
    off, ids, dist, _ = want
    assert np.array_equal(res.offsets, off), f"{label}: per-query counts differ"
    assert np.array_equal(res.ids, ids), f"{label}: ids differ"
    assert np.allclose(res.dist, dist, rtol=RTOL, atol=1e-30), f"{label}: angles beyond 1e-5 relative"


@pytest.mark.parametrize("dim,F", [(3, 6), (24, 7), (300, 8)])
def test_cos_range_and_knn(gts, dim, F):
    X, Q = cos_case(6000, dim, 48, seed=300 + dim)
    ix = gts.Index.build(X, "cos", fanout=F, root_pivot=1)
    radii = angle_radii(X, Q, 0.02, seed=7)
    radii[0] = 0.0                                   # exact direction matches only
    radii[1] = np.float32(np.pi)                     # every object
    radii[2] = np.float32(4.0)                       # beyond pi: every object too
    want_r = oracle.range_query("cos", X, Q, radii)
    ks = np.random.default_rng(dim).integers(1, 40, size=48).astype(np.int32)
    want_k = oracle.knn_query("cos", X, Q, ks)
    for prec in ("fp32", "bf16"):
        assert_same(ix.range(Q, radii, precision=prec), want_r, f"range d={dim} {prec}")
        r = ix.knn(Q, ks, precision=prec, keys=True)
        assert_same(r, want_k, f"knn d={dim} {prec}")
        assert np.array_equal(r.keys, want_k[3]), f"knn d={dim} {prec}: FP64 keys differ"
    ix.close()


def test_cos_rejects_zero_vectors(gts):
    X, Q = cos_case(500, 8, 4, seed=31)
    bad = X.copy()
    bad[17] = 0.0
    with pytest.raises(gts.GTSError):
        gts.Index.build(bad, "cos")
    ix = gts.Index.build(X, "cos")
    Qz = Q.copy()
    Qz[2] = 0.0
    with pytest.raises(gts.GTSError):
        ix.knn(Qz, 3)
    with pytest.raises(gts.GTSError):
        ix.insert(np.zeros((1, 8), np.float32))
    assert_same(ix.knn(Q, 3), oracle.knn_query("cos", X, Q, 3), "after rejected calls")
    ix.close()


@pytest.mark.parametrize("dim", [5, 64])
def test_cos_updates(gts, dim):
    """Inserts (the cache list keeps raw and unit rows), deletes, then a batch
    update (rebuild over the raw rows), each query against the oracle over the
    objects visible at its sequence number."""
    X, Q = cos_case(3000, dim, 20, seed=40 + dim)
    pool, _ = cos_case(600, dim, 1, seed=41 + dim)
    ix = gts.Index.build(X, "cos", fanout=6, root_pivot=0, cache_limit=150)
    n = X.shape[0]
    s0 = ix.info()["seq"]
    ids = ix.insert(pool[:100])
    assert list(ids) == list(range(n, n + 100))
    dele = np.random.default_rng(dim).choice(n + 100, 60, replace=False)
    assert ix.delete(dele) == 0
    P = np.concatenate([X, pool[:100]])
    ins = np.concatenate([np.full(n, -1), s0 + np.arange(100)]).astype(np.int64)
    dl = np.full(n + 100, np.iinfo(np.int64).max, np.int64)
    dl[dele] = s0 + 100 + np.arange(60)
    qs = np.full(20, ix.info()["seq"], np.int64)
    radii = angle_radii(P, Q, 0.03, seed=dim)
    assert_same(ix.range(Q, radii), oracle.range_query("cos", P, Q, radii, ins, dl, qs), "range after updates")
    assert_same(ix.knn(Q, 7), oracle.knn_query("cos", P, Q, 7, ins, dl, qs), "knn after updates")
    # a batch update rebuilds the tree from the raw rows
    s1 = ix.info()["seq"]
    live = np.setdiff1d(np.arange(n + 100), dele)
    victims = np.random.default_rng(dim + 1).choice(live, 30, replace=False)
    ids = ix.batch_update(pool[100:300], victims)
    assert list(ids) == list(range(n + 100, n + 300))
    P = np.concatenate([P, pool[100:300]])
    ins = np.concatenate([ins, s1 + np.arange(200)])
    dl = np.concatenate([dl, np.full(200, np.iinfo(np.int64).max, np.int64)])
    dl[victims] = s1 + 200 + np.arange(30)
    qs = np.full(20, ix.info()["seq"], np.int64)
    r = ix.knn(Q, 9, keys=True)
    want = oracle.knn_query("cos", P, Q, 9, ins, dl, qs)
    assert_same(r, want, "knn after batch update")
    assert np.array_equal(r.keys, want[3])
    ix.close()


def test_cos_save_load_round_trip(gts, tmp_path):
    X, Q = cos_case(4000, 40, 30, seed=55)
    extra, _ = cos_case(100, 40, 1, seed=56)
    ix = gts.Index.build(X, "cos", fanout=7, root_pivot=2, cache_limit=10_000)
    s0 = ix.info()["seq"]
    ix.insert(extra)
    path = str(tmp_path / "ix_cos.gts")
    ix.save(path)
    jx = gts.Index.load(path)
    assert jx.metric == "cos"
    assert jx.info() == {**ix.info(), "device_bytes": jx.info()["device_bytes"]}
    P = np.concatenate([X, extra])
    ins = np.concatenate([np.full(4000, -1), s0 + np.arange(100)]).astype(np.int64)
    dl = np.full(4100, np.iinfo(np.int64).max, np.int64)
    qs = np.full(30, ix.info()["seq"], np.int64)
    radii = angle_radii(P, Q, 0.02, seed=3)
    want_r = oracle.range_query("cos", P, Q, radii, ins, dl, qs)
    want_k = oracle.knn_query("cos", P, Q, 6, ins, dl, qs)
    for j in (ix, jx):
        assert_same(j.range(Q, radii), want_r, "range")
        r = j.knn(Q, 6, keys=True, precision="bf16")
        assert_same(r, want_k, "knn")
        assert np.array_equal(r.keys, want_k[3])
    ix.close()
    jx.close()


def test_cos_served_requests(gts):
    """The serving loop on an angular index: each request's answer equals the
    oracle's, and the admission projection bounds the candidates."""
    X, Q = cos_case(20000, 16, 60, seed=77)
    ix = gts.Index.build(X, "cos", fanout=8)
    sv = gts.Server(ix, max_batch=16, n_streams=2)
    radii = angle_radii(X, Q, 0.01, seed=5)
    kinds = ["range" if i % 2 else "knn" for i in range(60)]
    params = [float(radii[i]) if i % 2 else 5 for i in range(60)]
    tk = [sv.submit(Q[i], kinds[i], params[i]) for i in range(60)]
    got = [sv.wait(t) for t in tk]
    rows = [sv.project(Q[i], kinds[i], params[i]) // 37 for i in range(60)]
    sv.stop()
    want_r = oracle.range_query("cos", X, Q, radii)
    want_k = oracle.knn_query("cos", X, Q, 5)
    for i in range(60):
        off, wids, wdist, _ = want_r if i % 2 else want_k
        assert np.array_equal(got[i][0], wids[off[i]:off[i + 1]]), f"request {i}: ids differ from the oracle"
        assert np.allclose(got[i][1], wdist[off[i]:off[i + 1]], rtol=RTOL, atol=1e-30), f"request {i}: angles"
        assert rows[i] >= off[i + 1] - off[i], f"request {i}: projection below the answers"
    assert sum(r < X.shape[0] for r in rows[1::2]) > 0    # small angles prune some nodes
    ix.close()
