"""Multi-column queries through the C ABI (gts_multi_range / gts_multi_knn)
against the oracle's brute force over the summed distance (the closing remark
of Section 5.2: one index per column, pigeonhole principle for ranges,
Fagin's threshold algorithm for kNN).

Ids and offsets must match exactly and the FP64 sums bit for bit: every
column key is the single-column FP64 key, and both sides take sqrt and the C
library's acos of the same keys and add them in column order.

Inputs: three columns of one object set -- L2 over 24 dimensions, the angle
over 300 (the tensor-core tiles), L1 over 16 -- with duplicated objects (ties
broken by id), and a case whose columns disagree (independent data per
column, so the threshold algorithm needs several rounds of k' doubling).
"""
import numpy as np
import pytest

import oracle
from synth import small_vectors

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def gts():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2404_00966_gb300 import build_ext
    build_ext.build()
    import paper_2404_00966_gb300 as g
    return g


METRICS = ["l2", "cos", "l1"]
DIMS = [24, 300, 16]


def columns(n, nq, seed, correlated):
    """Per column (objects, queries); with ``correlated`` every column is a
    projection of one latent vector, so the columns rank objects alike."""
    rng = np.random.default_rng(seed)
    Xs, Qs = [], []
    latent, qlat = small_vectors(n, 8, nq, seed, kind="gauss", dup_frac=0.0)
    for j, d in enumerate(DIMS):
        if correlated:
            W = rng.standard_normal((8, d)).astype(np.float32)
            X = latent @ W + 0.05 * rng.standard_normal((n, d)).astype(np.float32)
            Q = qlat @ W + 0.05 * rng.standard_normal((nq, d)).astype(np.float32)
        else:
            X, Q = small_vectors(n, d, nq, seed + 17 * j + 1, kind="gauss", dup_frac=0.0)
        Xs.append(np.ascontiguousarray(X, np.float32))
        Qs.append(np.ascontiguousarray(Q, np.float32))
    dup = rng.choice(n, size=2 * (n // 50), replace=False)
    for X in Xs:                                              # the same objects duplicated in every column
        X[dup[: n // 50]] = X[dup[n // 50:]]
    for Q, X in zip(Qs, Xs):
        Q[0] = X[dup[0]]                                       # a query on a duplicated object
    return Xs, Qs


def sum_radii(Xs, Qs, frac, seed):
    rng = np.random.default_rng(seed)
    sample = rng.choice(Xs[0].shape[0], size=min(300, Xs[0].shape[0]), replace=False)
    S = [x[sample] for x in Xs]
    return np.array([np.quantile(oracle.multi_sums(METRICS, S, Qs, i), frac) for i in range(Qs[0].shape[0])],
                    np.float32)


def assert_same(res, want, label):
    off, ids, sums = want
    assert np.array_equal(res.offsets, off), f"{label}: per-query counts differ"
    assert np.array_equal(res.ids, ids), f"{label}: ids differ"
    assert np.array_equal(res.keys, sums), f"{label}: FP64 sums differ"
    assert np.array_equal(res.dist, sums.astype(np.float32)), f"{label}: FP32 distances differ"


@pytest.mark.parametrize("correlated", [True, False])
def test_multi_range_and_knn(gts, correlated):
    Xs, Qs = columns(5000, 40, seed=11 + correlated, correlated=correlated)
    cols = [gts.Index.build(X, m, fanout=8, root_pivot=3) for X, m in zip(Xs, METRICS)]
    radii = sum_radii(Xs, Qs, 0.01, seed=2)
    radii[0] = 0.0                                            # the duplicated object and its copy only
    radii[1] = np.float32(1e6)                                # every object
    want_r = oracle.multi_range(METRICS, Xs, Qs, radii)
    ks = np.random.default_rng(5).integers(1, 30, size=40).astype(np.int32)
    ks[2] = 1024                                              # the largest k
    want_k = oracle.multi_knn(METRICS, Xs, Qs, ks)
    for prec in ("fp32", "bf16"):
        rr = gts.multi_range(cols, Qs, radii, precision=prec)
        assert_same(rr, want_r, f"range {prec}")
        rk = gts.multi_knn(cols, Qs, ks, precision=prec)
        assert_same(rk, want_k, f"knn {prec}")
        for r, want in ((rr, want_r), (rk, want_k)):   # counters: the columns' searches summed
            assert r.stats["results"] == want[1].shape[0] and r.stats["table_pass"] == -1
            assert r.stats["launches"] > len(METRICS) and r.stats["pivot_dist"] > 0
    assert list(want_r[1][want_r[0][0]:want_r[0][1]]) == sorted(want_r[1][want_r[0][0]:want_r[0][1]])
    for c in cols:
        c.close()


def test_k_beyond_the_live_objects(gts):
    Xs, Qs = columns(700, 6, seed=51, correlated=False)
    cols = [gts.Index.build(X, m, fanout=5) for X, m in zip(Xs, METRICS)]
    ks = np.array([1000, 700, 699, 1, 1024, 350], np.int32)
    assert_same(gts.multi_knn(cols, Qs, ks), oracle.multi_knn(METRICS, Xs, Qs, ks), "k >= n")
    with pytest.raises(gts.GTSError):
        gts.multi_knn(cols, Qs, 1025)
    for c in cols:
        c.close()


def test_one_column_matches_the_single_column_oracle(gts):
    Xs, Qs = columns(3000, 25, seed=21, correlated=False)
    ix = gts.Index.build(Xs[2], "l1", fanout=10)
    got = gts.multi_knn([ix], [Qs[2]], 12)
    want = oracle.knn_query("l1", Xs[2], Qs[2], 12)
    assert np.array_equal(got.offsets, want[0]) and np.array_equal(got.ids, want[1])
    assert np.array_equal(got.keys, want[3])
    ix.close()


def test_multi_after_updates(gts):
    """Inserts and deletes applied to every column alike: the answers are the
    oracle's over the live objects."""
    Xs, Qs = columns(3000, 20, seed=31, correlated=True)
    extra, _ = columns(200, 1, seed=32, correlated=True)
    cols = [gts.Index.build(X, m, fanout=6, cache_limit=100) for X, m in zip(Xs, METRICS)]
    for c, e in zip(cols, extra):
        c.insert(e[:80])                                      # the cache list
    dele = np.random.default_rng(3).choice(3080, 90, replace=False)
    for c in cols:
        assert c.delete(dele) == 0
    for c, e in zip(cols, extra):
        c.batch_update(e[80:], np.zeros(0, np.int64))         # a rebuild
    P = [np.concatenate([X, e]) for X, e in zip(Xs, extra)]
    live = np.ones(3200, bool)
    live[dele] = False
    radii = sum_radii(P, Qs, 0.02, seed=4)
    assert_same(gts.multi_range(cols, Qs, radii), oracle.multi_range(METRICS, P, Qs, radii, live=live), "range")
    assert_same(gts.multi_knn(cols, Qs, 9), oracle.multi_knn(METRICS, P, Qs, 9, live=live), "knn")
    for c in cols:
        c.close()


def test_one_index_for_two_columns(gts):
    """The same index given twice (its columns run in turn): every distance
    doubles exactly, so the answers are the single column's at twice the
    distance -- and the oracle's duplicated-column sum."""
    Xs, Qs = columns(4000, 30, seed=61, correlated=False)
    a = gts.Index.build(Xs[0], "l2", fanout=9)
    got = gts.multi_knn([a, a], [Qs[0], Qs[0]], 8)
    assert_same(got, oracle.multi_knn(["l2", "l2"], [Xs[0], Xs[0]], [Qs[0], Qs[0]], 8), "knn")
    single = oracle.knn_query("l2", Xs[0], Qs[0], 8)
    assert np.array_equal(got.ids, single[1]) and np.array_equal(got.keys, 2.0 * single[2])
    radii = 2.0 * np.array([np.quantile(oracle.distances_to("l2", Xs[0], q), 0.01) for q in Qs[0]], np.float32)
    assert_same(gts.multi_range([a, a], [Qs[0], Qs[0]], radii),
                oracle.multi_range(["l2", "l2"], [Xs[0], Xs[0]], [Qs[0], Qs[0]], radii), "range")
    a.close()


def test_multi_device_queries(gts):
    """Device-resident query sets, radii and k give the host call's answers."""
    torch = pytest.importorskip("torch")
    Xs, Qs = columns(2000, 12, seed=81, correlated=True)
    cols = [gts.Index.build(X, m, fanout=7) for X, m in zip(Xs, METRICS)]
    Qd = [torch.from_numpy(q).cuda() for q in Qs]
    ks = np.arange(1, 13, dtype=np.int32)
    radii = sum_radii(Xs, Qs, 0.02, seed=9)
    assert_same(gts.multi_knn(cols, Qd, torch.from_numpy(ks).cuda()), oracle.multi_knn(METRICS, Xs, Qs, ks), "knn")
    assert_same(gts.multi_range(cols, Qd, torch.from_numpy(radii).cuda()),
                oracle.multi_range(METRICS, Xs, Qs, radii), "range")
    with pytest.raises(gts.GTSError):        # the sets on different sides
        gts.multi_knn(cols, [Qd[0], Qs[1], Qs[2]], 3)
    for c in cols:
        c.close()


def test_multi_empty_inputs(gts):
    """No queries; indexes with no objects; every object deleted."""
    Xs, Qs = columns(600, 5, seed=71, correlated=False)
    cols = [gts.Index.build(X, m, fanout=6) for X, m in zip(Xs, METRICS)]
    none = [q[:0] for q in Qs]
    for r in (gts.multi_knn(cols, none, 3), gts.multi_range(cols, none, np.zeros(0, np.float32))):
        assert list(r.offsets) == [0] and r.ids.size == 0
    for c in cols:
        c.delete(np.arange(600))
    r = gts.multi_knn(cols, Qs, 4)
    assert np.array_equal(r.offsets, np.zeros(6, np.int64)) and r.ids.size == 0
    r = gts.multi_range(cols, Qs, np.full(5, 1e6, np.float32))
    assert np.array_equal(r.offsets, np.zeros(6, np.int64))
    for c in cols:
        c.close()
    empty = [gts.Index.build(X[:0], m) for X, m in zip(Xs, METRICS)]
    r = gts.multi_knn(empty, Qs, 2)
    assert np.array_equal(r.offsets, np.zeros(6, np.int64))
    for c in empty:
        c.close()


def test_multi_argument_errors(gts):
    Xs, Qs = columns(800, 4, seed=41, correlated=False)
    a = gts.Index.build(Xs[0], "l2")
    b = gts.Index.build(Xs[2], "l1")
    with pytest.raises(gts.GTSError):                         # query dims swapped
        gts.multi_knn([a, b], [Qs[2], Qs[0]], 3)
    with pytest.raises(gts.GTSError):                         # different numbers of queries
        gts.multi_knn([a, b], [Qs[0], Qs[2][:2]], 3)
    with pytest.raises(ValueError):
        gts.multi_knn([a, b], [Qs[0]], 3)
    b.delete(np.array([5]))
    with pytest.raises(gts.GTSError):                         # live counts differ
        gts.multi_range([a, b], [Qs[0], Qs[2]], np.full(4, 1e6, np.float32))
    a.delete(np.array([6]))                                   # same counts, different ids
    with pytest.raises(gts.GTSError):
        gts.multi_range([a, b], [Qs[0], Qs[2]], np.full(4, 1e6, np.float32))
    c = gts.Index.build(Xs[2], "l1")
    r = gts.multi_knn([c], [Qs[2]], 3)                        # the library still answers after the errors
    assert np.array_equal(r.ids, oracle.knn_query("l1", Xs[2], Qs[2], 3)[1])
    for i in (a, b, c):
        i.close()
