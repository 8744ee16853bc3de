"""gts_knn_scan_noalloc: exact kNN by brute-force scan for callers that cannot
allocate device memory while they query (graph capture, allocator-free
serving threads, hosts that own all device memory).  Checked through the C
ABI against gts_knn on the same objects and against the CPU oracle, on two
calls in a row, so a second call that reuses the library's fixed scratch
array still answers exactly.

This file is collected last on purpose: a failure here comes after every other
test has run."""
import ctypes

import numpy as np
import pytest

import oracle
from synth import small_vectors

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


def _scan(g, torch, Xd, Qd, metric_id, k):
    nq, dim = Qd.shape
    ids = torch.empty(nq * k, dtype=torch.int64, device="cuda")
    dist = torch.empty(nq * k, dtype=torch.float32, device="cuda")
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    st = g.lib().gts_knn_scan_noalloc(ctypes.c_void_p(Xd.data_ptr()), Xd.shape[0], dim, metric_id,
                                      ctypes.c_void_p(Qd.data_ptr()), nq, k, ctypes.c_void_p(ids.data_ptr()),
                                      ctypes.c_void_p(dist.data_ptr()), stream)
    assert st == 0, g.lib().gts_last_error().decode()
    return ids.cpu().numpy().reshape(nq, k), dist.cpu().numpy().reshape(nq, k)


@pytest.mark.parametrize("metric,metric_id", [("l2", 2), ("l1", 1)])
def test_noalloc_scan_matches_gts_knn_on_two_calls(env, metric, metric_id):
    g, torch = env
    X, Q1 = small_vectors(6007, 48, 70, seed=91)
    _, Q2 = small_vectors(6007, 48, 45, seed=92)
    Q1[:2] = X[[3, 3]]                      # distance 0 and a duplicate query
    Xd = torch.from_numpy(X).cuda()
    ix = g.Index.build(Xd, metric, fanout=9, root_pivot=1)
    k = 12
    for Q in (Q1, Q2):                      # two calls in a row share the scratch array
        Qd = torch.from_numpy(Q).cuda()
        ids, dist = _scan(g, torch, Xd, Qd, metric_id, k)
        ref = ix.knn(Qd, k)
        off, wids, wdist, _ = oracle.knn_query(metric, X, Q, k)
        for i in range(Q.shape[0]):
            rid, rdist = ref.query(i)
            assert np.array_equal(ids[i], rid), f"query {i}: ids differ"
            assert np.allclose(dist[i], rdist, rtol=RTOL, atol=0), f"query {i}: distances differ"
            assert np.array_equal(ids[i], wids[off[i]:off[i + 1]]), f"query {i}: ids differ from the oracle"
            assert np.allclose(dist[i], wdist[off[i]:off[i + 1]], rtol=RTOL, atol=0), \
                f"query {i}: distances differ from the oracle"
    ix.close()


def test_noalloc_scan_nan_object_ranks_last(env):
    """A NaN coordinate makes that object's distance NaN; the scan ranks it as
    +inf, so the answers equal the oracle's over the other objects whenever k
    is at most their count."""
    g, torch = env
    X, Q = small_vectors(3001, 32, 40, seed=96)
    X[1234, 7] = np.nan
    keep = np.array([i for i in range(3001) if i != 1234])
    Xd, Qd = torch.from_numpy(X).cuda(), torch.from_numpy(Q).cuda()
    for metric, metric_id in (("l2", 2), ("l1", 1)):
        for _ in range(2):
            ids, dist = _scan(g, torch, Xd, Qd, metric_id, 16)
            off, wids, wdist, _ = oracle.knn_query(metric, X[keep], Q, 16)
            for i in range(40):
                assert np.array_equal(ids[i], keep[wids[off[i]:off[i + 1]]]), f"query {i}: ids differ"
                assert np.allclose(dist[i], wdist[off[i]:off[i + 1]], rtol=RTOL, atol=0)
    # three objects, one of them NaN, k = 3: the NaN object comes last at +inf
    Xs = np.array([[0.0, 1.0], [np.nan, 0.0], [2.0, 2.0]], np.float32)
    ids, dist = _scan(g, torch, torch.from_numpy(Xs).cuda(), torch.zeros((1, 2), device="cuda"), 2, 3)
    assert ids[0].tolist() == [0, 2, 1] and np.isinf(dist[0][2]) and dist[0][0] == 1.0


def test_noalloc_scan_fewer_objects_than_k_and_size_limit(env):
    g, torch = env
    X, Q = small_vectors(5, 8, 3, seed=93)
    Xd, Qd = torch.from_numpy(X).cuda(), torch.from_numpy(Q).cuda()
    ids, dist = _scan(g, torch, Xd, Qd, 2, 9)
    ix = g.Index.build(Xd, "l2", fanout=4)
    ref = ix.knn(Qd, 9)
    off, wids, wdist, _ = oracle.knn_query("l2", X, Q, 9)
    for i in range(3):
        rid, rdist = ref.query(i)
        assert np.array_equal(ids[i][:5], rid) and np.all(ids[i][5:] == -1)
        assert np.allclose(dist[i][:5], rdist, rtol=RTOL) and np.all(np.isinf(dist[i][5:]))
        assert np.array_equal(ids[i][:5], wids[off[i]:off[i + 1]])
    ix.close()
    # beyond the fixed scratch capacity: rejected with GTS_EINVAL, nothing launched
    st = g.lib().gts_knn_scan_noalloc(ctypes.c_void_p(Xd.data_ptr()), 5, 8, 2, ctypes.c_void_p(Qd.data_ptr()),
                                      (1 << 20) // 8 + 1, 8, ctypes.c_void_p(0), ctypes.c_void_p(0), None)
    assert st == 1 and b"scratch" in g.lib().gts_last_error()


def test_noalloc_scan_replayed_from_a_cuda_graph(env):
    """The asynchronous entry enqueues only its kernels, so a stream capture
    records it into a CUDA graph; replays with new query data in the same
    device buffer answer exactly."""
    g, torch = env
    X, Q1 = small_vectors(6007, 48, 64, seed=94)
    _, Q2 = small_vectors(6007, 48, 64, seed=95)
    Xd = torch.from_numpy(X).cuda()
    Qbuf = torch.from_numpy(Q1).cuda()
    k = 9
    ids = torch.empty(64 * k, dtype=torch.int64, device="cuda")
    dist = torch.empty(64 * k, dtype=torch.float32, device="cuda")
    _scan(g, torch, Xd, Qbuf, 2, k)   # the first call on the device looks up the scratch array, outside capture
    lib = g.lib()
    s = torch.cuda.Stream()
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph, stream=s):
        st = lib.gts_knn_scan_noalloc_async(ctypes.c_void_p(Xd.data_ptr()), Xd.shape[0], 48, 2,
                                            ctypes.c_void_p(Qbuf.data_ptr()), 64, k, ctypes.c_void_p(ids.data_ptr()),
                                            ctypes.c_void_p(dist.data_ptr()), ctypes.c_void_p(s.cuda_stream))
    assert st == 0, lib.gts_last_error().decode()
    ix = g.Index.build(Xd, "l2", fanout=9, root_pivot=1)
    for Q in (Q1, Q2):
        Qbuf.copy_(torch.from_numpy(Q))
        torch.cuda.synchronize()
        graph.replay()
        torch.cuda.synchronize()
        gi, gd = ids.cpu().numpy().reshape(64, k), dist.cpu().numpy().reshape(64, k)
        ref = ix.knn(Qbuf, k)
        off, wids, _, _ = oracle.knn_query("l2", X, Q, k)
        for i in range(64):
            rid, rdist = ref.query(i)
            assert np.array_equal(gi[i], rid), f"query {i}: ids differ"
            assert np.allclose(gd[i], rdist, rtol=RTOL, atol=0), f"query {i}: distances differ"
            assert np.array_equal(gi[i], wids[off[i]:off[i + 1]]), f"query {i}: ids differ from the oracle"
    ix.close()
