"""Continuous batching (gts_serve_*): every request's answer inside a mixed,
concurrently submitted stream equals its answer alone (gts_range / gts_knn on
that one query) and the CPU oracle's answer, and admission never lets the
projected bytes in flight exceed the budget (beyond one request admitted
alone)."""
import threading

import numpy as np
import pytest

import oracle
from synth import small_vectors, words_like

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


@pytest.mark.parametrize("metric,prec,quantum", [("l2", "fp32", 0), ("l2", "bf16", 0), ("l1", "fp32", 0),
                                                 ("l1", "bf16", 0), ("l1", "bf16", 4), ("l2", "bf16", 4)])
def test_mixed_stream_equals_alone(gts, metric, prec, quantum):
    X, Q = small_vectors(30011, 64, 240, seed=61)
    ix = gts.Index.build(X, metric, fanout=12, root_pivot=0)
    rng = np.random.default_rng(62)
    kinds = rng.random(240) < 0.5
    ks = rng.integers(1, 40, size=240)
    base = ix.knn(Q[:20], 30)
    radius = float(np.median([base.query(i)[1][-1] for i in range(20)]))
    proj = X.shape[0] * 37
    budget = 9 * proj                       # at most nine requests admitted at once
    sv = gts.Server(ix, max_batch=32, n_streams=3, precision=prec, result_budget=budget, batch_quantum=quantum)
    tickets = [None] * 240

    def submit(lo, hi):
        for i in range(lo, hi):
            tickets[i] = sv.submit(Q[i], "knn" if kinds[i] else "range", int(ks[i]) if kinds[i] else radius)

    th = [threading.Thread(target=submit, args=(a, a + 80)) for a in (0, 80, 160)]
    for t in th:
        t.start()
    for t in th:
        t.join()
    got = [sv.wait(t) for t in tickets]
    st = sv.stats()
    sv.stop()
    assert st["requests"] == 240 and st["batches"] > 1
    assert st["max_in_flight"] <= budget
    if quantum:   # batches above the quantum are cut to a multiple of it
        assert st["max_batch"] <= 4 or st["max_batch"] % quantum == 0
    want_k = oracle.knn_query(metric, X, Q, ks)
    want_r = oracle.range_query(metric, X, Q, np.full(240, radius, np.float32))
    for i in range(240):
        alone = ix.knn(Q[i:i + 1], int(ks[i]), precision=prec) if kinds[i] else \
            ix.range(Q[i:i + 1], np.float32([radius]), precision=prec)
        ids, dist = alone.query(0)
        assert np.array_equal(got[i][0], ids), f"request {i}: ids differ from the request alone"
        assert np.allclose(got[i][1], dist, rtol=1e-5, atol=1e-30), f"request {i}: distances differ"
        off, wids, wdist, _ = want_k if kinds[i] else want_r
        assert np.array_equal(got[i][0], wids[off[i]:off[i + 1]]), f"request {i}: ids differ from the oracle"
        assert np.allclose(got[i][1], wdist[off[i]:off[i + 1]], rtol=1e-5, atol=1e-30), \
            f"request {i}: distances differ from the oracle"
        assert got[i][2] >= 0.0
    ix.close()


def test_string_requests(gts):
    wl = words_like(n=3000, nq=60)
    ix = gts.Index.build(wl.objects, "edit", n_pivots=4, fanout=8, root_pivot=0)
    sv = gts.Server(ix, max_batch=16, n_streams=2)
    tk = [sv.submit(wl.queries.get(i), "range" if i % 2 else "knn", 2 if i % 2 else 5) for i in range(60)]
    got = [sv.wait(t) for t in tk]
    sv.stop()
    want_r = oracle.range_query("edit", wl.objects, wl.queries, np.full(60, 2, np.float32))
    want_k = oracle.knn_query("edit", wl.objects, wl.queries, 5)
    for i in range(60):
        q = wl.queries.take([i])
        alone = ix.range(q, np.float32([2])) if i % 2 else ix.knn(q, 5)
        ids, dist = alone.query(0)
        assert np.array_equal(got[i][0], ids) and np.array_equal(got[i][1], dist)
        off, wids, wdist, _ = want_r if i % 2 else want_k
        assert np.array_equal(got[i][0], wids[off[i]:off[i + 1]]), f"request {i}: ids differ from the oracle"
        assert np.array_equal(got[i][1], wdist[off[i]:off[i + 1]].astype(np.float32))
    ix.close()


@pytest.mark.parametrize("metric", ["l2", "l1"])
def test_admission_projection_bounds_the_candidates(gts, metric):
    """The projection (host descent over the top pivot levels) is an upper
    bound of every request's candidates: for a range request at least the
    pairs that pass the table bound in the full search of that request alone,
    for kNN at least its answers (the nodes it keeps hold the ball of radius
    d_k); on clustered data with a small radius it is below the worst case."""
    X, Q = small_vectors(40009, 4, 60, seed=63)
    ix = gts.Index.build(X, metric, fanout=6, root_pivot=0)
    d = np.sort(oracle.distances_to(metric, X[:2000], Q[0]))
    radius = float(d[20])
    sv = gts.Server(ix, max_batch=8, n_streams=1)
    below = 0
    for i in range(60):
        for kind, param in (("range", radius), ("knn", 5)):
            rows = sv.project(Q[i], kind, param) // 37
            alone = ix.range(Q[i:i + 1], np.float32([param]), count_table_pass=True) if kind == "range" else \
                ix.knn(Q[i:i + 1], int(param), count_table_pass=True)
            assert rows >= alone.offsets[1], (i, kind)
            if kind == "range":
                assert rows >= alone.stats["table_pass"], i
            below += rows < 40009
    sv.stop()
    assert below >= 60    # the range requests at least: a small radius prunes most nodes
    ix.close()
