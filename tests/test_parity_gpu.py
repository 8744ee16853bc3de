"""Parity of the CUDA path (through the C ABI) with the CPU oracle on seeded
inputs that span several tiles, ragged tails and the degenerate cases.

Bar: edit distance bit-exact (ids and integer distances); L1 / L2 identical id
sets (the FP64 boundary recheck decides every close call exactly as the
oracle does) and distances within 1e-5 relative of the oracle's FP64 value.
"""
import numpy as np
import pytest

import oracle
from oracle.index import build_index
from synth import Strings, mutate, random_strings, small_vectors, strings_from_list, words_like

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


def assert_same(res, want, metric, label=""):
    off, ids, dist, _ = want
    assert np.array_equal(res.offsets, off), f"{label}: per-query counts differ"
    assert np.array_equal(res.ids, ids), f"{label}: ids differ"
    if metric == "edit":
        assert np.array_equal(res.dist, dist.astype(np.float32)), f"{label}: edit distances differ"
    else:
        assert np.allclose(res.dist, dist, rtol=RTOL, atol=1e-30), f"{label}: distances beyond 1e-5 relative"


def vec_case(n, dim, nq, seed, kind="gauss", dup=0.0):
    return small_vectors(n, dim, nq, seed, kind=kind, dup_frac=dup)


def str_case(n, nq, seed, lmin=1, lmax=20, alphabet=b"abcd"):
    rng = np.random.default_rng(seed)
    alpha = np.frombuffer(alphabet, np.uint8)
    S = random_strings(n, lmin, lmax, alpha, rng)
    qs = [mutate(S.get(int(rng.integers(0, n))), int(rng.integers(0, 4)), alpha, rng) for _ in range(nq)]
    return S, strings_from_list(qs)


# ------------------------------------------------------------------ index build

@pytest.mark.parametrize("metric,F,npiv", [("l2", 6, 0), ("l1", 5, 3), ("edit", 8, 4)])
def test_build_matches_oracle_tree(gts, metric, F, npiv):
    if metric == "edit":
        objs, _ = str_case(2500, 1, seed=1)
    else:
        objs, _ = vec_case(3001, 24, 1, seed=2, dup=0.1)
    ix = gts.Index.build(objs, metric, n_pivots=npiv, fanout=F, root_pivot=11)
    T = build_index(objs, metric, F, npiv, root_pivot=11)
    info = ix.info()
    assert info["h"] == T["h"]
    for l in range(T["h"] + 1):
        g = ix.tree_level(l)
        assert np.array_equal(g["pos"], T["pos"][l]) and np.array_equal(g["size"], T["size"][l])
        if l >= 1:
            assert np.array_equal(g["lo"], T["lo"][l]) and np.array_equal(g["hi"], T["hi"][l])
        if l < T["h"]:
            assert np.array_equal(g["pivot"], T["pivot"][l])
    ids, tab = ix.table()
    assert np.array_equal(ids, T["perm"])
    assert np.array_equal(tab, T["table"])
    ix.close()


@pytest.mark.parametrize("metric", ["l1", "l2"])
def test_build_matches_oracle_tree_with_exact_ties(gts, metric):
    """Integer points in a small cube: exactly tied distances at every level,
    so the (distance, id) order of the partition decides every cut."""
    X = np.random.default_rng(5).integers(0, 3, size=(2400, 3)).astype(np.float32)
    ix = gts.Index.build(X, metric, n_pivots=3, fanout=6, root_pivot=7)
    T = build_index(X, metric, 6, 3, root_pivot=7)
    for l in range(T["h"] + 1):
        g = ix.tree_level(l)
        assert np.array_equal(g["pos"], T["pos"][l]) and np.array_equal(g["size"], T["size"][l])
        if l < T["h"]:
            assert np.array_equal(g["pivot"], T["pivot"][l])
    ids, tab = ix.table()
    assert np.array_equal(ids, T["perm"])
    assert np.array_equal(tab, T["table"])
    ix.close()


# ------------------------------------------------------------------ range / kNN parity

@pytest.mark.parametrize("metric", ["l2", "l1"])
@pytest.mark.parametrize("dup", [0.0, 0.3])
def test_vector_range_and_knn(gts, metric, dup):
    X, Q = vec_case(5003, 40, 97, seed=3, dup=dup)
    Q[:5] = X[[0, 17, 17, 4000, 5002]]                      # exact copies: distance 0 and ties
    ix = gts.Index.build(X, metric, fanout=7, root_pivot=3)
    d = oracle.distances_to(metric, X[:400], Q[7])
    base = float(np.median(d))
    radii = np.concatenate([[0.0, 0.0], np.linspace(0.3, 1.2, 95) * base]).astype(np.float32)
    assert_same(ix.range(Q, radii), oracle.range_query(metric, X, Q, radii), metric, "range")
    for k in (1, 10, 57):
        assert_same(ix.knn(Q, k), oracle.knn_query(metric, X, Q, k), metric, f"knn k={k}")
    ks = np.random.default_rng(4).integers(1, 100, size=97).astype(np.int32)
    assert_same(ix.knn(Q, ks), oracle.knn_query(metric, X, Q, ks), metric, "knn mixed k")
    ix.close()


@pytest.mark.parametrize("prec", ["fp32", "bf16"])   # bf16: the 3-gram filtering tiles
def test_edit_range_and_knn(gts, prec):
    S, Qs = str_case(4000, 80, seed=5)
    ix = gts.Index.build(S, "edit", n_pivots=4, fanout=8, root_pivot=1)
    radii = np.random.default_rng(6).integers(0, 5, size=80).astype(np.float32) + 0.7
    r = ix.range(Qs, radii, precision=prec)
    assert (r.stats["tiles"] > 0) == (prec == "bf16")
    assert_same(r, oracle.range_query("edit", S, Qs, radii), "edit", "range")
    for k in (1, 5, 40):
        assert_same(ix.knn(Qs, k, precision=prec), oracle.knn_query("edit", S, Qs, k), "edit", f"knn k={k}")
    ix.close()


def test_edit_long_strings_multiword(gts):
    """Lengths above 64 and 128 (several 64-bit words per bit-parallel column)."""
    rng = np.random.default_rng(7)
    alpha = np.frombuffer(b"ACGT", np.uint8)
    seeds = random_strings(40, 60, 300, alpha, rng)
    items = [mutate(seeds.get(i % 40), int(rng.integers(0, 12)), alpha, rng) for i in range(1200)]
    S = strings_from_list(items)
    Qs = strings_from_list([mutate(seeds.get(int(rng.integers(0, 40))), int(rng.integers(0, 8)), alpha, rng)
                            for _ in range(30)])
    ix = gts.Index.build(S, "edit", fanout=6, root_pivot=0)
    radii = np.full(30, 10.0, np.float32)
    want_r = oracle.range_query("edit", S, Qs, radii)
    want_k = oracle.knn_query("edit", S, Qs, 12)
    for prec in ("fp32", "bf16"):
        assert_same(ix.range(Qs, radii, precision=prec), want_r, "edit", f"long range {prec}")
        assert_same(ix.knn(Qs, 12, precision=prec), want_k, "edit", f"long knn {prec}")
    ix.close()


def test_words_like_full_size(gts):
    """The 10,000-string / 256-query / radius-2 workload, every query checked."""
    wl = words_like()
    ix = gts.Index.build(wl.objects, "edit", n_pivots=wl.n_pivots, fanout=wl.fanout, root_pivot=0)
    want = oracle.range_query("edit", wl.objects, wl.queries, wl.radii)
    for prec in ("fp32", "bf16"):
        assert_same(ix.range(wl.queries, wl.radii, precision=prec), want, "edit", f"words {prec}")
    ix.close()


# ------------------------------------------------------------------ degenerate cases

def test_empty_and_tiny(gts):
    X = np.zeros((0, 8), np.float32)
    ix = gts.Index.build(X, "l2", fanout=4)
    Q = np.ones((3, 8), np.float32)
    r = ix.range(Q, np.ones(3, np.float32))
    assert list(r.offsets) == [0, 0, 0, 0]
    r = ix.knn(Q, 2)
    assert list(r.offsets) == [0, 0, 0, 0]
    ix.close()
    X1 = np.arange(8, dtype=np.float32)[None, :]
    ix = gts.Index.build(X1, "l1", fanout=4)
    assert_same(ix.knn(Q, 5), oracle.knn_query("l1", X1, Q, 5), "l1", "n=1")
    r = ix.range(np.zeros((0, 8), np.float32), np.zeros(0, np.float32))
    assert list(r.offsets) == [0]
    ix.close()


def test_all_identical_objects(gts):
    X = np.tile(np.float32([[0.5, -1.0, 2.0]]), (777, 1))
    Q = np.float32([[0.5, -1.0, 2.0], [1.5, -1.0, 2.0]])
    ix = gts.Index.build(X, "l2", fanout=5, root_pivot=0)
    assert_same(ix.knn(Q, 33), oracle.knn_query("l2", X, Q, 33), "l2", "identical knn")
    assert_same(ix.range(Q, np.float32([0.0, 1.0])), oracle.range_query("l2", X, Q, np.float32([0.0, 1.0])), "l2",
                "identical range")
    ix.close()


def test_empty_strings_and_short(gts):
    items = [b"", b"a", b"b", b"ab", b"", b"abc", b"ba"] * 30
    S = strings_from_list(items)
    Qs = strings_from_list([b"", b"a", b"abcd"])
    ix = gts.Index.build(S, "edit", fanout=3, root_pivot=2)
    radii = np.float32([0, 1, 2])
    assert_same(ix.range(Qs, radii), oracle.range_query("edit", S, Qs, radii), "edit", "short range")
    assert_same(ix.knn(Qs, 9), oracle.knn_query("edit", S, Qs, 9), "edit", "short knn")
    ix.close()


def test_k_larger_than_n(gts):
    X, Q = vec_case(300, 5, 4, seed=9)
    ix = gts.Index.build(X, "l2", fanout=4)
    assert_same(ix.knn(Q, 1000), oracle.knn_query("l2", X, Q, 1000), "l2", "k>n")
    ix.close()


def test_invalid_arguments(gts):
    X, Q = vec_case(200, 5, 3, seed=10)
    ix = gts.Index.build(X, "l2", fanout=4)
    with pytest.raises(gts.GTSError) as e:
        ix.range(Q, np.float32([1, -1, 1]))
    assert e.value.name == "GTS_EINVAL"
    with pytest.raises(gts.GTSError):
        ix.range(Q, np.float32([1, np.nan, 1]))
    with pytest.raises(gts.GTSError):
        ix.knn(Q, 0)
    Qbad = Q.copy()
    Qbad[1, 2] = np.inf
    with pytest.raises(gts.GTSError):
        ix.knn(Qbad, 3)
    with pytest.raises(gts.GTSError):
        ix.knn(np.zeros((2, 6), np.float32), 3)
    ix.close()


# ------------------------------------------------------------------ scheduler, precision, residency

def test_tiny_memory_budget_gives_same_answers(gts):
    X, Q = vec_case(6000, 16, 150, seed=11)
    ix = gts.Index.build(X, "l1", fanout=8)
    radii = np.full(150, np.float32(np.median(oracle.distances_to("l1", X[:300], Q[0])) * 0.6))
    want_r = oracle.range_query("l1", X, Q, radii)
    want_k = oracle.knn_query("l1", X, Q, 9)
    r = ix.range(Q, radii, memory_budget=64 << 10)
    assert r.stats["groups"] > 1
    assert_same(r, want_r, "l1", "budget range")
    assert_same(ix.knn(Q, 9, memory_budget=64 << 10), want_k, "l1", "budget knn")
    ix.close()


def _bf16(x):
    """Round float32 to bfloat16 (nearest, ties to even) and back, in numpy."""
    u = np.ascontiguousarray(x, np.float32).view(np.uint32).astype(np.uint64)
    r = ((u + 0x7FFF + ((u >> 16) & 1)) & 0xFFFF0000).astype(np.uint32)
    return r.view(np.float32)


@pytest.mark.parametrize("a_tmem", [False, True])
@pytest.mark.parametrize("N,K", [(256, 128), (64, 64), (128, 256), (32, 192)])
def test_tensor_core_tile_primitives(gts, N, K, a_tmem):
    """TMA (128-byte swizzle) + tcgen05.mma (TMEM accumulator) + tcgen05.ld,
    with A from shared memory or from TMEM (tcgen05.st, two coordinates per
    column), against the FP64 product of the same bf16-rounded inputs."""
    rng = np.random.default_rng(N * 1000 + K)
    A = rng.standard_normal((128, K)).astype(np.float32)
    B = rng.standard_normal((N, K)).astype(np.float32)
    D = gts.selftest_tc(A, B, a_tmem=a_tmem)
    ref = _bf16(A).astype(np.float64) @ _bf16(B).astype(np.float64).T
    scale = np.abs(_bf16(A)).astype(np.float64) @ np.abs(_bf16(B)).astype(np.float64).T
    err = np.abs(D - ref)
    assert np.all(err <= (K + 4) * 2.0 ** -23 * scale + 1e-30), float((err / scale).max())


def test_bounded_wait_runs_out_and_device_stays_usable(gts):
    """A wait on an mbarrier that nothing arrives on gives up after its poll
    limit: the kernel records the run-out and returns, the call reports
    GTS_ETIMEOUT, and the device answers the next query exactly."""
    L = gts.lib()
    assert L.gts_selftest_wait(0, 1 << 14) == 4                 # GTS_ETIMEOUT
    assert b"ran out" in L.gts_last_error()
    assert L.gts_selftest_wait(1, 1 << 14) == 0                 # posted: the wait ends
    assert L.gts_selftest_wait(0, 0) == 1                       # limit out of range: GTS_EINVAL
    X, Q = vec_case(2003, 16, 20, seed=31)
    ix = gts.Index.build(X, "l2", fanout=6, root_pivot=2)
    assert_same(ix.knn(Q, 5), oracle.knn_query("l2", X, Q, 5), "l2", "after a run-out")
    ix.close()


@pytest.mark.parametrize("dim,dup", [(128, 0.0), (100, 0.2), (256, 0.0), (300, 0.1), (384, 0.0), (448, 0.0)])
def test_bf16_tiles_parity(gts, dim, dup):
    """Every tile shape: 128 queries per chunk (dim <= 128), 64 (dim_p 192 and
    320), 32 (dim_p 256, 384 and 448)."""
    X, Q = vec_case(20011, dim, 300, seed=40 + dim, dup=dup)
    Q[:3] = X[[5, 9, 20010]]
    ix = gts.Index.build(X, "l2", fanout=12, root_pivot=7)
    assert ix.knn(Q[:4], 3, precision="bf16").stats["tiles"] > 0     # the tensor-core tiles run
    for k in (1, 10, 33):
        r = ix.knn(Q, k, precision="bf16")
        assert_same(r, oracle.knn_query("l2", X, Q, k), "l2", f"bf16 tiles knn k={k}")
    d = oracle.distances_to("l2", X[:500], Q[4])
    # wide frontiers: dense pivot matrices and (128-query tiles) the dense last level
    wide = ix.knn(Q, 500, precision="bf16")
    assert wide.stats["dense_pairs"] > 0 and wide.stats["dense_last"] == (1 if dim <= 128 else 0)
    assert_same(wide, oracle.knn_query("l2", X, Q, 500), "l2", "bf16 tiles knn k=500 (dense last level)")
    big = np.full(300, np.float32(np.median(d)), np.float32)
    rb = ix.range(Q, big, precision="bf16")
    assert rb.stats["dense_last"] == (1 if dim <= 128 else 0)
    assert_same(rb, oracle.range_query("l2", X, Q, big), "l2", "bf16 tiles wide range (dense last level)")
    radii = np.linspace(0.0, 1.0, 300).astype(np.float32) * np.float32(np.median(d))
    assert_same(ix.range(Q, radii, precision="bf16"), oracle.range_query("l2", X, Q, radii), "l2", "bf16 tiles range")
    ix.close()


@pytest.mark.parametrize("dim,kind,dup", [(64, "gauss", 0.0), (100, "gauss", 0.2), (256, "uniform", 0.0)])
def test_l1_tiles_parity(gts, dim, kind, dup):
    """L1 node-major FP32 tiles (precision="bf16" selects them for L1): blocks
    of several 128-row slices, chunks of more than 128 queries, a coordinate
    tail (dim 100), exact copies and ties, kNN run in three phases."""
    X, Q = vec_case(20011, dim, 300, seed=50 + dim, kind=kind, dup=dup)
    Q[:3] = X[[5, 9, 20010]]
    ix = gts.Index.build(X, "l1", fanout=12, root_pivot=7)
    for k in (1, 10, 57):
        r = ix.knn(Q, k, precision="bf16")
        assert r.stats["tile_pairs"] > 0
        assert_same(r, oracle.knn_query("l1", X, Q, k), "l1", f"L1 tiles knn k={k}")
    ks = np.random.default_rng(5).integers(1, 100, size=300).astype(np.int32)
    assert_same(ix.knn(Q, ks, precision="bf16"), oracle.knn_query("l1", X, Q, ks), "l1", "L1 tiles knn mixed k")
    d = oracle.distances_to("l1", X[:500], Q[4])
    radii = np.linspace(0.0, 0.9, 300).astype(np.float32) * np.float32(np.median(d))
    assert_same(ix.range(Q, radii, precision="bf16"), oracle.range_query("l1", X, Q, radii), "l1", "L1 tiles range")
    ix.close()


def test_l1_tiles_concentrated_distances(gts):
    """Uniform 128-d data: the lower bounds prune almost nothing, every block
    holds every query, and the kNN phases must lower tau from the probe's."""
    X, Q = vec_case(30011, 128, 260, seed=61, kind="uniform")
    ix = gts.Index.build(X, "l1", fanout=20, root_pivot=0)
    for k in (1, 100):
        r = ix.knn(Q, k, precision="bf16")
        assert r.stats["dense_pairs"] > 0           # the per-level dense pivot matrices ran
        assert_same(r, oracle.knn_query("l1", X, Q, k), "l1", f"concentrated knn k={k}")
    cal = oracle.knn_query("l1", X, Q[:10], 30)
    radii = np.full(260, np.float32(np.mean(cal[2][cal[0][1:] - 1])), np.float32)
    assert_same(ix.range(Q, radii, precision="bf16"), oracle.range_query("l1", X, Q, radii), "l1", "concentrated range")
    ix.close()


def test_low_dim_takes_the_table_scan(gts):
    X, Q = vec_case(3000, 6, 40, seed=62)
    ix = gts.Index.build(X, "l1", fanout=6)
    r = ix.knn(Q, 5, precision="bf16")
    assert r.stats["tile_pairs"] == 0 and r.stats["scanned_rows"] > 0
    assert_same(r, oracle.knn_query("l1", X, Q, 5), "l1", "dim 6")
    ix.close()


@pytest.mark.parametrize("metric", ["l2", "l1"])
@pytest.mark.parametrize("dim", [2, 3, 8, 16])
def test_scan_low_dim_parity(gts, metric, dim):
    """Node-major table scan + CUDA-core verification (precision="bf16" on
    vectors of dim <= 16): duplicates and exact ties, radius 0, a ragged last
    block, every k from 1 to past the 64-record chunk."""
    X, Q = vec_case(20011, dim, 300, seed=90 + dim, dup=0.2)
    Q[:3] = X[[5, 9, 20010]]
    ix = gts.Index.build(X, metric, fanout=8, root_pivot=3)
    d = oracle.distances_to(metric, X[:500], Q[4])
    radii = np.concatenate([[0.0, 0.0], np.linspace(0.01, 0.3, 298) * np.median(d)]).astype(np.float32)
    r = ix.range(Q, radii, precision="bf16", count_table_pass=True)
    assert r.stats["scanned_rows"] > 0 and r.stats["tile_pairs"] == 0
    # the scan emits exactly the pairs that pass the table bound
    assert r.stats["table_pass"] == r.stats["candidates"]
    assert_same(r, oracle.range_query(metric, X, Q, radii), metric, f"scan range dim {dim}")
    for k in (1, 10, 90):
        assert_same(ix.knn(Q, k, precision="bf16"), oracle.knn_query(metric, X, Q, k), metric,
                    f"scan knn k={k} dim {dim}")
    ix.close()


def test_scan_many_blocks_and_chunks_and_relaunch(gts):
    """Two pivot levels of fanout 4 over 20,000 2-D points: last-level nodes of
    5,000 rows (40 row blocks each) with hundreds of query records (several
    64-record chunks); a wide radius emits more candidates than the first
    launch's capacity (1 M), so the scan runs again with the exact size."""
    X, Q = vec_case(20000, 2, 600, seed=97, kind="uniform")
    ix = gts.Index.build(X, "l2", n_pivots=2, fanout=4, root_pivot=1)
    radii = np.full(600, 0.25, np.float32)
    r = ix.range(Q, radii, precision="bf16")
    assert r.stats["candidates"] > (1 << 20)
    assert_same(r, oracle.range_query("l2", X, Q, radii), "l2", "wide radius")
    small = np.full(600, 0.02, np.float32)
    assert_same(ix.range(Q, small, precision="bf16"), oracle.range_query("l2", X, Q, small), "l2", "small radius")
    assert_same(ix.knn(Q, 33, precision="bf16"), oracle.knn_query("l2", X, Q, 33), "l2", "knn 33")
    ix.close()


@pytest.mark.parametrize("metric", ["l2", "l1"])
def test_scan_with_stream_updates(gts, metric):
    """Inserts in the cache list and deletes of tree rows and cache objects:
    the scan skips deleted rows by their sequence numbers."""
    X, Q = vec_case(30011, 2, 200, seed=98)
    ix = gts.Index.build(X, metric, fanout=12, root_pivot=0, cache_limit=100_000)
    s0 = ix.info()["seq"]
    extra, _ = vec_case(700, 2, 1, seed=99)
    ix.insert(extra)
    dele = np.random.default_rng(100).choice(30011 + 700, 2000, replace=False)
    assert ix.delete(dele) == 0
    s1 = ix.info()["seq"]
    P = np.concatenate([X, extra])
    ins = np.concatenate([np.full(30011, -1), s0 + np.arange(700)]).astype(np.int64)
    dl = np.full(P.shape[0], np.iinfo(np.int64).max, np.int64)
    dl[dele] = s0 + 700 + np.arange(2000)
    qs = np.full(200, s1, np.int64)
    d = oracle.distances_to(metric, X[:300], Q[0])
    radii = np.full(200, np.float32(np.median(d) * 0.1), np.float32)
    r = ix.range(Q, radii, precision="bf16")
    assert r.stats["scanned_rows"] > 0
    assert_same(r, oracle.range_query(metric, P, Q, radii, ins, dl, qs), metric, "scan range with updates")
    assert_same(ix.knn(Q, 12, precision="bf16"), oracle.knn_query(metric, P, Q, 12, ins, dl, qs), metric,
                "scan knn with updates")
    ix.close()


@pytest.mark.parametrize("metric,dim", [("l2", 32), ("l1", 3)])
def test_shape_autotuner_keeps_answers(gts, metric, dim):
    """gts_autotune_shape ranks (fanout, h) by the cost model, rebuilds and
    times the cheapest shapes and keeps the fastest: the index ends in that
    shape, and every shape it timed answers exactly."""
    X, Q = vec_case(30011, dim, 200, seed=130 + dim)
    ix = gts.Index.build(X, metric, fanout=20, root_pivot=0)
    want = oracle.knn_query(metric, X, Q, 10)
    d = oracle.distances_to(metric, X[:300], Q[0])
    radii = np.full(200, np.float32(np.median(d) * 0.2), np.float32)
    want_r = oracle.range_query(metric, X, Q, radii)
    shapes = ix.autotune_shape(Q, k=10, precision="bf16", candidates=3, reps=1)
    assert 3 <= len(shapes) <= 4
    ms = [sh["measured_ms"] for sh in shapes]
    assert ms == sorted(ms) and all(m > 0 for m in ms)
    info = ix.info()
    assert (info["fanout"], info["h"]) == (shapes[0]["fanout"], shapes[0]["n_pivots"])
    assert_same(ix.knn(Q, 10, precision="bf16"), want, metric, "after shape tuning")
    assert_same(ix.range(Q, radii, precision="bf16"), want_r, metric, "range after shape tuning")
    for sh in shapes:
        j = gts.Index.build(X, metric, n_pivots=sh["n_pivots"], fanout=sh["fanout"], root_pivot=0)
        assert_same(j.knn(Q, 10, precision="bf16"), want, metric, f"shape {sh}")
        assert_same(j.range(Q, radii, precision="fp32"), want_r, metric, f"shape {sh} range")
        j.close()
    ix.close()


@pytest.mark.parametrize("prec,dim", [("fp32", 32), ("bf16", 64), ("bf16", 128)])
def test_table_pass_count_is_consistent(gts, prec, dim):
    """The diagnostic count of pairs passing the table bound: on the plain
    path it equals the scan's candidates; on the tensor-core tiles it is at
    most the pairs the tiles covered; the answers do not change."""
    X, Q = vec_case(20011, dim, 200, seed=120 + dim)
    ix = gts.Index.build(X, "l2", fanout=12, root_pivot=5)
    want = oracle.knn_query("l2", X, Q, 10)
    r = ix.knn(Q, 10, precision=prec, count_table_pass=True)
    assert_same(r, want, "l2", "knn with the count")
    assert ix.knn(Q, 10, precision=prec).stats["table_pass"] == -1
    if prec == "fp32":
        assert r.stats["table_pass"] == r.stats["candidates"]
    else:
        assert 0 < r.stats["table_pass"] <= r.stats["tile_pairs"]
    ix.close()


@pytest.mark.parametrize("metric,prec", [("l1", "bf16"), ("l2", "bf16"), ("l2", "fp32")])
def test_every_tuning_gives_the_same_answers(gts, metric, prec):
    X, Q = vec_case(12007, 64, 150, seed=71, kind="uniform" if metric == "l1" else "gauss")
    ix = gts.Index.build(X, metric, fanout=10, root_pivot=2)
    ks = np.random.default_rng(72).integers(1, 60, size=150).astype(np.int32)
    want = oracle.knn_query(metric, X, Q, ks)
    cal = oracle.knn_query(metric, X, Q[:5], 20)
    radii = np.full(150, np.float32(np.mean(cal[2][cal[0][1:] - 1])), np.float32)
    want_r = oracle.range_query(metric, X, Q, radii)
    for lq in (64, 128):
        for packed in (0, 1):
            for phases in (1, 2, 3):
                for probe in (0, 256, 4096):
                    if metric != "l1" and (lq, packed, phases) != (128, 1, 3) and (lq, packed, phases, probe) != (
                            64, 0, 1, 256):
                        continue
                    # the (64, 0, 1, 256) setting of L2 also takes the 96-query, 3-slot tensor-core tiles
                    tcq = 96 if (lq, packed, phases, probe) == (64, 0, 1, 256) else 128
                    ix.set_tuning(l1_queries=lq, l1_packed=packed, knn_phases=phases, probe_rows=probe,
                                  tc_queries=tcq)
                    tag = f"{lq}/{packed}/{phases}/{probe}"
                    assert_same(ix.knn(Q, ks, precision=prec), want, metric, f"knn tuning {tag}")
                    if probe == 0:
                        assert_same(ix.range(Q, radii, precision=prec), want_r, metric, f"range tuning {tag}")
    with pytest.raises(gts.GTSError):
        ix.set_tuning(knn_phases=4)
    with pytest.raises(gts.GTSError):
        ix.set_tuning(tc_queries=100)
    t = ix.autotune(Q, k=ks, precision=prec, reps=1)
    assert t["tuned"] == 1 and t["l1_queries"] in (64, 128) and 0 <= t["probe_rows"] <= 4096
    assert t["tc_queries"] in (96, 128)
    assert ix.get_tuning() == t
    assert_same(ix.knn(Q, ks, precision=prec), want, metric, "after autotune")
    t2 = ix.autotune(Q, radii=radii, precision=prec, reps=1)
    assert t2["tuned"] == 1
    assert_same(ix.range(Q, radii, precision=prec), want_r, metric, "after range autotune")
    ix.close()


def test_bf16_tiles_deep_tree(gts):
    """Ten pivot levels: the tile's per-query path distances do not fit three
    staging slots, so the kernel runs two slots of 128 queries."""
    X, Q = vec_case(6007, 64, 160, seed=81)
    ix = gts.Index.build(X, "l2", n_pivots=10, fanout=3, root_pivot=0)
    assert ix.info()["h"] == 10
    ix.set_tuning(tc_queries=96)   # asks for three slots of 96; the kernel falls back to two of 128
    for k in (1, 7):
        assert_same(ix.knn(Q, k, precision="bf16"), oracle.knn_query("l2", X, Q, k), "l2", f"deep tree knn k={k}")
    d = oracle.distances_to("l2", X[:300], Q[1])
    radii = np.linspace(0.0, 0.8, 160).astype(np.float32) * np.float32(np.median(d))
    assert_same(ix.range(Q, radii, precision="bf16"), oracle.range_query("l2", X, Q, radii), "l2", "deep tree range")
    ix.close()


def test_bf16_precision_same_answers(gts):
    X, Q = vec_case(8000, 64, 120, seed=12)
    ix = gts.Index.build(X, "l2", fanout=10)
    want = oracle.knn_query("l2", X, Q, 10)
    assert_same(ix.knn(Q, 10, precision="bf16"), want, "l2", "bf16 knn")
    radii = np.full(120, 1.0, np.float32)
    assert_same(ix.range(Q, radii, precision="bf16"), oracle.range_query("l2", X, Q, radii), "l2", "bf16 range")
    ix.close()


def test_device_inputs_and_results(gts):
    import torch
    X, Q = vec_case(4000, 32, 50, seed=13)
    Xd, Qd = torch.from_numpy(X).cuda(), torch.from_numpy(Q).cuda()
    ix = gts.Index.build(Xd, "l2", fanout=9)
    k = torch.full((50,), 6, dtype=torch.int32, device="cuda")
    res = ix.knn(Qd, k, result_on_device=True)
    host = ix.knn(Qd, k)
    want = oracle.knn_query("l2", X, Q, 6)
    assert_same(host, want, "l2", "device inputs")
    tot = int(want[0][-1])
    t_off = torch.empty(51, dtype=torch.int64, device="cuda")
    t_ids = torch.empty(tot, dtype=torch.int64, device="cuda")
    t_dist = torch.empty(tot, dtype=torch.float32, device="cuda")
    res.copy_to(t_off, t_ids, t_dist)
    assert np.array_equal(t_off.cpu().numpy(), want[0])
    assert np.array_equal(t_ids.cpu().numpy(), want[1])
    res.free()
    ix.close()


# ------------------------------------------------------------------ updates

def _replay(gts, metric, objs_init, pool, seed, cache_limit, precision="fp32"):
    """Insert / delete / query interleaving (Section 4.4) checked against the
    oracle over the objects visible at each query's sequence number."""
    rng = np.random.default_rng(seed)
    is_str = isinstance(objs_init, Strings)
    ix = gts.Index.build(objs_init, metric, fanout=6, root_pivot=0, cache_limit=cache_limit)
    n0 = objs_init.n if is_str else objs_init.shape[0]
    all_items = [objs_init.get(i) for i in range(n0)] if is_str else list(objs_init)
    ins = [-1] * n0
    dele = [np.iinfo(np.int64).max] * n0
    live = list(range(n0))
    seq = ix.info()["seq"]
    p = 0
    for step in range(12):
        # inserts
        m = int(rng.integers(1, 9))
        new = pool[p:p + m]
        p += m
        newobj = strings_from_list(new) if is_str else np.asarray(new, np.float32)
        ids = ix.insert(newobj)
        assert list(ids) == list(range(len(all_items), len(all_items) + m))
        for j in range(m):
            all_items.append(new[j])
            ins.append(seq)
            dele.append(np.iinfo(np.int64).max)
            seq += 1
        live += list(ids)
        # deletes (one unknown id on purpose)
        victims = list(rng.choice(live, size=min(len(live), int(rng.integers(1, 6))), replace=False))
        missing = ix.delete(np.array(victims + [10 ** 7], np.int64))
        assert missing == 1
        for v in victims:
            dele[v] = seq
            seq += 1
            live.remove(v)
        assert ix.info()["seq"] == seq
        # queries at the current state
        if is_str:
            Qs = strings_from_list([mutate(all_items[int(rng.integers(0, len(all_items)))], 1,
                                           np.frombuffer(b"abcd", np.uint8), rng) for _ in range(7)])
            P = strings_from_list(all_items)
        else:
            Qs = np.asarray([all_items[int(rng.integers(0, len(all_items)))] for _ in range(7)], np.float32) + 0.01
            P = np.asarray(all_items, np.float32)
        qseq = np.full(7, seq, np.int64)
        I, Dl = np.asarray(ins, np.int64), np.asarray(dele, np.int64)
        radii = np.full(7, 2.0 if is_str else 0.8, np.float32)
        assert_same(ix.range(Qs, radii, precision=precision), oracle.range_query(metric, P, Qs, radii, I, Dl, qseq),
                    metric, f"update range step {step}")
        assert_same(ix.knn(Qs, 5, precision=precision), oracle.knn_query(metric, P, Qs, 5, I, Dl, qseq), metric,
                    f"update knn {step}")
    # batch update = rebuild
    newb = pool[p:p + 40]
    newobj = strings_from_list(newb) if is_str else np.asarray(newb, np.float32)
    victims = list(rng.choice(live, size=10, replace=False))
    ids = ix.batch_update(newobj, np.array(victims, np.int64))
    for j in range(len(newb)):
        all_items.append(newb[j])
        ins.append(seq)
        dele.append(np.iinfo(np.int64).max)
        seq += 1
    for v in victims:
        dele[v] = seq
        seq += 1
    inf = ix.info()
    assert inf["n_cache"] == 0 and inf["rebuild_seq"] == seq == inf["seq"]
    P = strings_from_list(all_items) if is_str else np.asarray(all_items, np.float32)
    Qs = P.take(np.arange(5)) if is_str else P[:5]
    qseq = np.full(5, seq, np.int64)
    I, Dl = np.asarray(ins, np.int64), np.asarray(dele, np.int64)
    assert_same(ix.knn(Qs, 8, precision=precision), oracle.knn_query(metric, P, Qs, 8, I, Dl, qseq), metric,
                "after batch update")
    ix.close()


@pytest.mark.parametrize("cache_limit", [1, 7, 10000])
def test_updates_vectors(gts, cache_limit):
    X, _ = vec_case(1500, 6, 1, seed=14)
    pool, _ = vec_case(400, 6, 1, seed=15)
    _replay(gts, "l2", X, list(pool), seed=16, cache_limit=cache_limit)


@pytest.mark.parametrize("precision", ["fp32", "bf16"])
def test_updates_vectors_l1(gts, precision):
    X, _ = vec_case(1500, 8, 1, seed=24)
    pool, _ = vec_case(400, 8, 1, seed=25)
    _replay(gts, "l1", X, list(pool), seed=26, cache_limit=7, precision=precision)


@pytest.mark.parametrize("prec", ["fp32", "bf16"])
def test_updates_strings(gts, prec):
    S, _ = str_case(1200, 1, seed=17, lmin=2, lmax=10)
    P, _ = str_case(400, 1, seed=18, lmin=2, lmax=10)
    _replay(gts, "edit", S, [P.get(i) for i in range(P.n)], seed=19, cache_limit=9, precision=prec)


def test_query_sequence_numbers_span_updates(gts):
    """One batch whose queries see different states (per-query seq)."""
    X, Q = vec_case(2000, 8, 6, seed=20)
    ix = gts.Index.build(X, "l1", fanout=6)
    s0 = ix.info()["seq"]
    extra, _ = vec_case(30, 8, 1, seed=21)
    ix.insert(extra)
    ix.delete(np.arange(0, 200, 7))
    s1 = ix.info()["seq"]
    P = np.concatenate([X, extra])
    ins = np.concatenate([np.full(2000, -1), s0 + np.arange(30)]).astype(np.int64)
    dele = np.full(2030, np.iinfo(np.int64).max, np.int64)
    dele[np.arange(0, 200, 7)] = s0 + 30 + np.arange(len(range(0, 200, 7)))
    qseq = np.array([s0, s0 + 10, s0 + 30, s0 + 35, s1, s1], np.int64)
    assert_same(ix.knn(Q, 7, seq=qseq), oracle.knn_query("l1", P, Q, 7, ins, dele, qseq), "l1", "seq knn")
    ix.close()


# ------------------------------------------------------------------ persistence and shards

@pytest.mark.parametrize("metric", ["l2", "edit"])
def test_save_load_round_trip(gts, tmp_path, metric):
    """An index written by gts_save and read by gts_load answers exactly as
    the saved one, cache list, delete marks and sequence numbers included;
    updates continue on the loaded index."""
    if metric == "edit":
        X, Q = str_case(3000, 40, seed=140)
        extra, _ = str_case(200, 1, seed=141)
        radii = np.full(40, 2.0, np.float32)
    else:
        X, Q = vec_case(8000, 24, 40, seed=140, dup=0.1)
        extra, _ = vec_case(200, 24, 1, seed=141)
        radii = np.full(40, np.float32(np.median(oracle.distances_to("l2", X[:200], Q[0])) * 0.5), np.float32)
    ix = gts.Index.build(X, metric, fanout=7, root_pivot=3, cache_limit=10_000)
    s0 = ix.info()["seq"]
    ix.insert(extra)
    n = 3000 if metric == "edit" else 8000
    dele = np.random.default_rng(142).choice(n + 200, 300, replace=False)
    assert ix.delete(dele) == 0
    path = str(tmp_path / f"ix_{metric}.gts")
    ix.save(path)
    jx = gts.Index.load(path)
    assert jx.info() == {**ix.info(), "device_bytes": jx.info()["device_bytes"]}
    if metric == "edit":
        P = strings_from_list([X.get(i) for i in range(n)] + [extra.get(i) for i in range(200)])
    else:
        P = np.concatenate([X, extra])
    ins = np.concatenate([np.full(n, -1), s0 + np.arange(200)]).astype(np.int64)
    dl = np.full(n + 200, np.iinfo(np.int64).max, np.int64)
    dl[dele] = s0 + 200 + np.arange(300)
    qs = np.full(40, ix.info()["seq"], np.int64)
    want_r = oracle.range_query(metric, P, Q, radii, ins, dl, qs)
    want_k = oracle.knn_query(metric, P, Q, 9, ins, dl, qs)
    for j in (ix, jx):
        for prec in ("fp32", "bf16"):
            assert_same(j.range(Q, radii, precision=prec), want_r, metric, f"range {prec}")
            r = j.knn(Q, 9, precision=prec, keys=True)
            assert_same(r, want_k, metric, f"knn {prec}")
            assert np.array_equal(r.keys, want_k[3])              # the exact FP64 (or integer) keys
    ids = jx.insert(extra)                                        # updates continue on the loaded index
    assert ids[0] == n + 200
    ix.close()
    jx.close()


@pytest.mark.parametrize("metric", ["l2", "l1"])
def test_sharded_index_equals_one_index(gts, metric):
    """Objects split into three shards (one index each), every query sent to
    every shard, answers merged by gts_merge_*: the same answers as the
    oracle over the union, exact ties across shards included."""
    rng = np.random.default_rng(150)
    X = rng.integers(0, 5, size=(9001, 4)).astype(np.float32)
    Q = rng.integers(0, 5, size=(60, 4)).astype(np.float32)
    sh = gts.ShardedIndex.build(X, metric, 3, fanout=6, root_pivot=0)
    ks = rng.integers(1, 50, size=60).astype(np.int32)
    for prec in ("fp32", "bf16"):
        assert_same(sh.knn(Q, ks, precision=prec), oracle.knn_query(metric, X, Q, ks), metric, f"shards knn {prec}")
        radii = np.full(60, 2.0, np.float32)
        assert_same(sh.range(Q, radii, precision=prec), oracle.range_query(metric, X, Q, radii), metric,
                    f"shards range {prec}")
    sh.close()


def test_every_string_tuning_gives_the_same_answers(gts):
    """Edit distance: every DP block size and 3-gram filter setting (off, 32 or
    64 queries per chunk) answers exactly; the autotuner searches them."""
    S, Qs = str_case(5000, 90, seed=160, lmin=6, lmax=40)
    ix = gts.Index.build(S, "edit", n_pivots=3, fanout=8, root_pivot=2)
    radii = np.random.default_rng(161).integers(0, 6, size=90).astype(np.float32)
    want_r = oracle.range_query("edit", S, Qs, radii)
    want_k = oracle.knn_query("edit", S, Qs, 7)
    for chunk in (64, 128, 256, 512):
        for qg in (0, 32, 64):
            ix.set_tuning(str_chunk=chunk, str_qgram=qg)
            r = ix.range(Qs, radii, precision="bf16")
            assert (r.stats["tiles"] > 0) == (qg > 0)
            assert_same(r, want_r, "edit", f"range chunk {chunk} qgram {qg}")
            assert_same(ix.knn(Qs, 7, precision="bf16"), want_k, "edit", f"knn chunk {chunk} qgram {qg}")
    with pytest.raises(gts.GTSError):
        ix.set_tuning(str_chunk=100)
    with pytest.raises(gts.GTSError):
        ix.set_tuning(str_qgram=16)
    t = ix.autotune(Qs, radii=radii, precision="bf16", reps=1)
    assert t["str_chunk"] in (64, 128, 256, 512) and t["str_qgram"] in (0, 32, 64)
    assert_same(ix.range(Qs, radii, precision="bf16"), want_r, "edit", "after autotune")
    ix.close()
