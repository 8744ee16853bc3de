"""Pins of the oracle's multi-column definition (the closing remark of
Section 5.2: one index per column, the distance of an object the sum of its
column distances).  Each pin holds by the mathematics, not by the oracle's own
code:

* one column: the summed distance is that column's distance, so the answers
  are the single-column oracle's (itself pinned elsewhere);
* L1 over a split of the coordinates: the sum of the parts' L1 distances is
  the L1 distance of the whole vector (up to FP64 summation order);
* a duplicated column: the sum is exactly twice the column distance;
* an L2 column and an angular column over the same unit vectors: the sum is
  2 sin(theta / 2) + theta for the angle theta between them;
* the sum of metrics is a metric: symmetric, zero on duplicates, triangle
  inequality; ties in the kNN order are broken by the smaller id.
"""
import math

import numpy as np
import pytest

import oracle


def gauss(n, dim, seed):
    return np.random.default_rng(seed).standard_normal((n, dim)).astype(np.float32)


def test_one_column_is_the_column_itself():
    X, Q = gauss(500, 12, 1), gauss(10, 12, 2)
    off, ids, sums = oracle.multi_knn(["l1"], [X], [Q], 9)
    w = oracle.knn_query("l1", X, Q, 9)
    assert np.array_equal(off, w[0]) and np.array_equal(ids, w[1])
    assert np.array_equal(sums, w[3])                         # 0 + key is exact
    radii = np.array([np.quantile(oracle.distances_to("l1", X, q), 0.05) for q in Q], np.float32)
    off, ids, _ = oracle.multi_range(["l1"], [X], [Q], radii)
    w = oracle.range_query("l1", X, Q, radii)
    assert np.array_equal(off, w[0]) and np.array_equal(ids, w[1])


def test_l1_split_columns_sum_to_the_whole():
    X, Q = gauss(800, 20, 3), gauss(12, 20, 4)
    cols, qs = [X[:, :7], X[:, 7:15], X[:, 15:]], [Q[:, :7], Q[:, 7:15], Q[:, 15:]]
    off, ids, sums = oracle.multi_knn(["l1"] * 3, cols, qs, 15)
    w = oracle.knn_query("l1", X, Q, 15)
    assert np.array_equal(ids, w[1])
    assert np.allclose(sums, w[2], rtol=1e-12)


def test_duplicated_column_doubles_the_distance():
    X, Q = gauss(600, 9, 5), gauss(8, 9, 6)
    off, ids, sums = oracle.multi_knn(["l2", "l2"], [X, X], [Q, Q], 11)
    w = oracle.knn_query("l2", X, Q, 11)
    assert np.array_equal(ids, w[1])
    assert np.array_equal(sums, 2.0 * w[2])                  # sqrt(key) + sqrt(key), exact
    radii = np.array([np.quantile(oracle.distances_to("l2", X, q), 0.03) for q in Q], np.float32)
    off, ids, _ = oracle.multi_range(["l2", "l2"], [X, X], [Q, Q], 2.0 * radii)
    w = oracle.range_query("l2", X, Q, radii)
    assert np.array_equal(off, w[0]) and np.array_equal(ids, w[1])


def test_chord_plus_angle_on_unit_vectors():
    U = gauss(300, 5, 7).astype(np.float64)
    U /= np.linalg.norm(U, axis=1, keepdims=True)
    U = U.astype(np.float32)
    q = U[:3]
    for i in range(3):
        s = oracle.multi_sums(["l2", "cos"], [U, U], [q, q], i)
        a, b = q[i].astype(np.float64), U.astype(np.float64)
        theta = np.arccos(np.clip(b @ a / (np.linalg.norm(b, axis=1) * np.linalg.norm(a)), -1, 1))
        assert np.allclose(s, 2.0 * np.sin(theta / 2.0) + theta, rtol=0, atol=2e-6)


def test_metric_properties_and_tie_order():
    X = gauss(60, 6, 8)
    X[30:40] = X[:10]                                         # duplicates: sum 0 between them
    Y = gauss(60, 4, 9)
    Y[30:40] = Y[:10]
    mets = ["l2", "l1"]
    D = np.array([oracle.multi_sums(mets, [X, Y], [X, Y], i) for i in range(60)])
    assert np.allclose(D, D.T, rtol=1e-12, atol=0)
    assert np.all(np.diag(D) == 0.0) and np.all(D[np.arange(10), np.arange(30, 40)] == 0.0)
    for i in range(0, 60, 7):
        for j in range(0, 60, 5):
            assert np.all(D[i, j] <= D[i, :] + D[:, j] + 1e-9)
    off, ids, sums = oracle.multi_knn(mets, [X, Y], [X[:10], Y[:10]], 3)
    for i in range(10):                                       # the row and its duplicate tie at 0
        assert list(ids[off[i]:off[i] + 2]) == [i, 30 + i] and sums[off[i]] == sums[off[i] + 1] == 0.0
    off, ids, _ = oracle.multi_range(mets, [X, Y], [X[:10], Y[:10]], np.zeros(10, np.float32))
    assert all(list(ids[off[i]:off[i + 1]]) == [i, 30 + i] for i in range(10))   # <= r holds at r = 0


def test_live_mask_and_k_beyond_n():
    X, Q = gauss(50, 4, 10), gauss(3, 4, 11)
    live = np.ones(50, bool)
    live[::3] = False
    off, ids, _ = oracle.multi_knn(["l2"], [X], [Q], 100, live=live)
    assert np.all(np.diff(off) == live.sum()) and live[ids].all()
    off, ids, _ = oracle.multi_range(["l2"], [X], [Q], np.full(3, np.inf, np.float32), live=live)
    assert np.all(np.diff(off) == live.sum())
    with pytest.raises(ValueError):
        oracle.column_distances("edit", X, Q[0])
    # the C loop calls the same function as math.acos
    keys = oracle.keys_to_pivot("cos", np.concatenate([X, -X[:1]]), 0)
    ang = oracle.column_distances("cos", np.concatenate([X, -X[:1]]), X[0])
    assert all(ang[i] == math.acos(1.0 - keys[i]) for i in range(keys.shape[0]))
    # antipodal rows: pi, up to acos's sqrt-like sensitivity at -1 to the FP64 rounding of cos
    assert math.isclose(oracle.column_distances("cos", -X[:1], X[0])[0], math.pi, rel_tol=0, abs_tol=1e-7)


def test_knn_is_the_range_at_its_kth_sum():
    """Definitions 1 and 2 over the summed distance agree: a query's k nearest
    are the range answers at its k-th sum, up to ties at that sum (which the
    kNN order breaks by id)."""
    X, Q = gauss(700, 5, 12), gauss(9, 5, 13)
    Y, R = gauss(700, 3, 14), gauss(9, 3, 15)
    mets = ["l1", "l2"]
    off, ids, sums = oracle.multi_knn(mets, [X, Y], [Q, R], 17)
    radii = np.array([sums[off[i + 1] - 1] for i in range(9)], np.float32)
    roff, rids, rsums = oracle.multi_range(mets, [X, Y], [Q, R], np.nextafter(radii, np.float32(np.inf)))
    for i in range(9):
        ki, ks = ids[off[i]:off[i + 1]], sums[off[i]:off[i + 1]]
        ri, rs = rids[roff[i]:roff[i + 1]], rsums[roff[i]:roff[i + 1]]
        assert set(ki) <= set(ri)                                 # every kNN answer is inside the radius
        assert np.all(rs[~np.isin(ri, ki)] >= ks[-1])             # the rest are no nearer than the k-th
        assert np.all(np.diff(ks) >= 0)
