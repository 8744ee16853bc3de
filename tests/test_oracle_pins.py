"""Pins of the CPU oracle against facts that do not come from the oracle:
exhaustive search over edit sequences, hand-checked textbook pairs, closed
forms, exact rational arithmetic, metric axioms and brute-force subset checks
of Definitions 1 and 2 (Section 3).  CPU only."""
import itertools
import os
from collections import deque
from fractions import Fraction

import numpy as np
import pytest

import oracle
from oracle.index import build_index, height
from synth import Strings, strings_from_list

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


# ------------------------------------------------------------ edit distance

def _bfs_distances(src: str, alphabet: str, maxlen: int) -> dict:
    """Edit distance as its definition: the least number of single-character
    insertions, deletions and substitutions turning ``src`` into each string,
    found by breadth-first search over strings of length <= maxlen."""
    dist = {src: 0}
    dq = deque([src])
    while dq:
        s = dq.popleft()
        nbrs = set()
        for i in range(len(s)):
            nbrs.add(s[:i] + s[i + 1:])
            for c in alphabet:
                if c != s[i]:
                    nbrs.add(s[:i] + c + s[i + 1:])
        if len(s) < maxlen:
            for i in range(len(s) + 1):
                for c in alphabet:
                    nbrs.add(s[:i] + c + s[i:])
        for t in nbrs:
            if t not in dist:
                dist[t] = dist[s] + 1
                dq.append(t)
    return dist


def test_edit_full_matches_exhaustive_search():
    alphabet = "ab"
    strs = [""] + ["".join(p) for L in range(1, 5) for p in itertools.product(alphabet, repeat=L)]
    for a in strs:
        bfs = _bfs_distances(a, alphabet, 5)
        for b in strs:
            assert oracle.edit_full(a.encode(), b.encode()) == bfs[b], (a, b)


def test_edit_golden_pairs():
    n = 0
    with open(os.path.join(GOLDEN, "edit_pairs.txt")) as f:
        for line in f:
            if line.startswith("#") or not line.strip():
                continue
            a, b, d, _src = line.rstrip("\n").split("\t")
            a = "" if a == "<empty>" else a
            b = "" if b == "<empty>" else b
            assert oracle.edit_full(a.encode(), b.encode()) == int(d), (a, b)
            n += 1
    assert n >= 10


def test_edit_banded_equals_capped_full():
    rng = np.random.default_rng(7)
    for _ in range(20000):
        la, lb = rng.integers(0, 14, size=2)
        a = bytes(rng.choice(list(b"acgt"), size=la).tolist())
        b = bytes(rng.choice(list(b"acgt"), size=lb).tolist())
        r = int(rng.integers(0, 9))
        full = oracle.edit_full(a, b)
        assert oracle.edit_banded(a, b, r) == min(full, r + 1), (a, b, r)


def test_edit_banded_long_strings():
    rng = np.random.default_rng(8)
    for _ in range(300):
        base = bytes(rng.choice(list(b"ACGT"), size=108).tolist())
        other = bytearray(base)
        for _e in range(int(rng.integers(0, 14))):
            p = int(rng.integers(0, len(other)))
            other[p] = int(rng.choice(list(b"ACGT")))
        r = int(rng.integers(0, 12))
        assert oracle.edit_banded(base, bytes(other), r) == min(oracle.edit_full(base, bytes(other)), r + 1)


def test_edit_metric_axioms():
    rng = np.random.default_rng(9)
    pool = [bytes(rng.choice(list(b"abc"), size=int(rng.integers(0, 9))).tolist()) for _ in range(40)]
    for x in pool:
        assert oracle.edit_full(x, x) == 0
    for x, y, z in itertools.islice(itertools.product(pool, repeat=3), 0, 64000, 7):
        dxy, dyz, dxz = oracle.edit_full(x, y), oracle.edit_full(y, z), oracle.edit_full(x, z)
        assert dxy == oracle.edit_full(y, x)
        assert dxz <= dxy + dyz
        assert dxy >= abs(len(x) - len(y))
        if x != y:
            assert dxy > 0


# ------------------------------------------------------------ L1 / L2

def test_l2_l1_closed_forms():
    D = 128
    a = np.zeros(D, np.float32)
    b = np.zeros(D, np.float32)
    b[0], b[D - 1] = 3.0, -4.0           # the last coordinate carries a term
    assert oracle.l2sq(a, b) == 25.0
    assert oracle.l1(a, b) == 7.0
    assert oracle.l2sq(b, a) == 25.0
    # a single coordinate: |x - y| exactly
    c = np.zeros(D, np.float32)
    c[D - 1] = 0.5
    assert oracle.l1(a, c) == 0.5 and oracle.l2sq(a, c) == 0.25
    # power-of-two scaling is exact
    rng = np.random.default_rng(3)
    x = rng.standard_normal(D).astype(np.float32)
    y = rng.standard_normal(D).astype(np.float32)
    assert oracle.l2sq(2 * x, 2 * y) == 4 * oracle.l2sq(x, y)
    assert oracle.l1(4 * x, 4 * y) == 4 * oracle.l1(x, y)
    assert oracle.l2sq(x, x) == 0.0 and oracle.l1(x, x) == 0.0


def test_l2_l1_against_exact_rationals():
    rng = np.random.default_rng(4)
    for D in (1, 2, 3, 17, 128, 256):
        for _ in range(20):
            x = (rng.standard_normal(D) * rng.choice([1e-3, 1, 1e3])).astype(np.float32)
            y = (rng.standard_normal(D) * rng.choice([1e-3, 1, 1e3])).astype(np.float32)
            ex2 = sum((Fraction(float(p)) - Fraction(float(q))) ** 2 for p, q in zip(x, y))
            ex1 = sum(abs(Fraction(float(p)) - Fraction(float(q))) for p, q in zip(x, y))
            # recursive summation of D non-negative terms: relative error <= gamma_{D+1}
            u = 2.0 ** -53
            g = (D + 1) * u / (1 - (D + 1) * u)
            assert abs(Fraction(oracle.l2sq(x, y)) - ex2) <= Fraction(g) * ex2
            assert abs(Fraction(oracle.l1(x, y)) - ex1) <= Fraction(g) * ex1


def test_vector_metric_axioms():
    rng = np.random.default_rng(5)
    P = rng.standard_normal((30, 16)).astype(np.float32)
    for i, j, k in itertools.product(range(30), repeat=3):
        if (i * 31 + j * 7 + k) % 5:
            continue
        for f, sq in ((oracle.l2sq, True), (oracle.l1, False)):
            dij, djk, dik = (f(P[i], P[j]), f(P[j], P[k]), f(P[i], P[k]))
            if sq:
                dij, djk, dik = np.sqrt(dij), np.sqrt(djk), np.sqrt(dik)
            assert dij == (np.sqrt(f(P[j], P[i])) if sq else f(P[j], P[i]))
            assert dik <= (dij + djk) * (1 + 1e-12)


# ------------------------------------------------------------ angular (cosine) distance

def test_cos_closed_forms():
    """Norms chosen exact (3-4-5 triangles): c and the key exactly."""
    e1, e2 = np.float32([1, 0, 0]), np.float32([0, 1, 0])
    assert oracle.cos_key(e1, e2) == 1.0                       # orthogonal: pi / 2
    x = np.float32([3, 4])
    assert oracle.cos_key(x, 4 * x) == 0.0                     # one direction: angle 0
    assert oracle.cos_key(x, np.float32([-1.5, -2])) == 2.0    # opposite: angle pi
    assert oracle.cos_key(np.float32([3, 4]), np.float32([4, 3])) == 1.0 - 24.0 / 25.0
    assert oracle.cos_key(np.float32([3, 4, 0]), np.float32([0, 4, 3])) == 1.0 - 16.0 / 25.0
    # 45 degrees: c = 1/sqrt(2) within rounding
    assert abs(oracle.cos_key(np.float32([1, 0]), np.float32([1, 1])) - (1 - 2 ** -0.5)) < 4e-16
    # the range limit: 1 - cos(r), r clipped at pi
    assert oracle.cos_limit(0.0) == 0.0
    assert oracle.cos_limit(4.0) == 2.0 and oracle.cos_limit(np.pi) == oracle.cos_limit(4.0)
    assert abs(oracle.cos_limit(np.pi / 2) - 1.0) < 1e-7       # float32(pi / 2) is not pi / 2
    # distances
    d = oracle.distances_to("cos", np.float32([[3, 4], [4, 3], [-3, -4]]), np.float32([3, 4]))
    assert d[0] == 0.0 and abs(d[1] - np.arccos(24 / 25)) < 1e-15 and d[2] == np.pi


def test_cos_scaling_axioms_and_long_double():
    rng = np.random.default_rng(6)
    D = 300
    P = rng.standard_normal((24, D)).astype(np.float32)
    for i in range(24):
        for j in range(24):
            k = oracle.cos_key(P[i], P[j])
            # power-of-two scaling changes no rounding: the same key
            assert oracle.cos_key(4 * P[i], 0.25 * P[j]) == k
            assert k == oracle.cos_key(P[j], P[i])               # symmetry
            a, b = P[i].astype(np.longdouble), P[j].astype(np.longdouble)
            c = (a @ b) / (np.sqrt(a @ a) * np.sqrt(b @ b))
            # three recursive sums and a few roundings: well within 4 (D + 4) 2^-53
            assert abs(k - float(1 - c)) <= 4 * (D + 4) * 2.0 ** -53
    ang = lambda u, v: float(np.arccos(1.0 - oracle.cos_key(u, v)))
    for i, j, k in itertools.product(range(12), repeat=3):
        assert ang(P[i], P[k]) <= ang(P[i], P[j]) + ang(P[j], P[k]) + 1e-12
    assert all(oracle.cos_key(P[i], P[i]) <= 4e-16 for i in range(24))


def _exact_cos_order(X, q):
    """A key with the same order as the cosine, in exact rationals:
    sign(q.x) (q.x)^2 / |x|^2 (|q| is common to all x)."""
    out = []
    for x in X:
        dot = sum(Fraction(float(a)) * Fraction(float(b)) for a, b in zip(q, x))
        nx = sum(Fraction(float(b)) ** 2 for b in x)
        out.append((1 if dot > 0 else (-1 if dot < 0 else 0)) * dot * dot / nx)
    return out


def test_range_and_knn_cos_by_exhaustion():
    """Integer points: many exactly equal angles.  Range: exactly the objects
    whose exact cosine clears cos(r) (radii kept off every object's angle);
    kNN: k members, none of them with a smaller exact cosine than a
    non-member, in (FP64 key, id) order."""
    rng = np.random.default_rng(13)
    n, D, nq = 150, 4, 12
    X = rng.integers(-3, 4, size=(n, D)).astype(np.float32)
    X[np.all(X == 0, axis=1)] = 1.0                             # no zero vector
    Q = rng.integers(-3, 4, size=(nq, D)).astype(np.float32)
    Q[np.all(Q == 0, axis=1)] = 1.0
    ks = rng.integers(1, 20, size=nq).astype(np.int32)
    radii = np.float32(rng.uniform(0.2, 2.5, size=nq))
    off, ids, dist, keys = oracle.range_query("cos", X, Q, radii)
    koff, kids, kdist, kkeys = oracle.knn_query("cos", X, Q, ks)
    for qi in range(nq):
        q = Q[qi]
        nq2 = float(q.astype(np.float64) @ q.astype(np.float64))
        cos_exact = [float(q.astype(np.float64) @ x.astype(np.float64)) / np.sqrt(nq2 * float(x.astype(np.float64) @ x.astype(np.float64))) for x in X]
        cr = np.cos(np.float64(radii[qi]))
        assert min(abs(c - cr) for c in cos_exact) > 1e-9       # no object on the boundary
        want = [o for o in range(n) if cos_exact[o] > cr]
        assert list(ids[off[qi]:off[qi + 1]]) == want
        ex = _exact_cos_order(X, q)
        got = list(kids[koff[qi]:koff[qi + 1]])
        assert len(got) == min(int(ks[qi]), n)
        outside = [o for o in range(n) if o not in got]
        assert min(ex[s] for s in got) >= max(ex[o] for o in outside)
        assert list(kkeys[koff[qi]:koff[qi + 1]]) == sorted(kkeys[koff[qi]:koff[qi + 1]])


# ------------------------------------------------------------ range / kNN sets

def _exact_keys_vec(metric, X, q):
    out = []
    for x in X:
        if metric == "l2":
            out.append(sum((Fraction(float(a)) - Fraction(float(b))) ** 2 for a, b in zip(q, x)))
        else:
            out.append(sum(abs(Fraction(float(a)) - Fraction(float(b))) for a, b in zip(q, x)))
    return out


@pytest.mark.parametrize("metric", ["l1", "l2"])
def test_range_and_knn_vectors_by_exhaustion(metric):
    rng = np.random.default_rng(11)
    n, D, nq = 120, 6, 12
    X = rng.integers(-3, 4, size=(n, D)).astype(np.float32)   # small integers: many exact ties
    Q = rng.integers(-3, 4, size=(nq, D)).astype(np.float32)
    radii = rng.integers(0, 6, size=nq).astype(np.float32)
    ks = rng.integers(1, 15, size=nq).astype(np.int32)
    off, ids, dist, keys = oracle.range_query(metric, X, Q, radii)
    koff, kids, kdist, kkeys = oracle.knn_query(metric, X, Q, ks)
    for qi in range(nq):
        ex = _exact_keys_vec(metric, X, Q[qi])
        r = Fraction(float(radii[qi]))
        lim = r * r if metric == "l2" else r
        want = [o for o in range(n) if ex[o] <= lim]
        assert list(ids[off[qi]:off[qi + 1]]) == want
        # Definition 2 by exhaustion: the answer has k members, every member is
        # no farther than every non-member, and it is the (key, id)-first set.
        got = list(kids[koff[qi]:koff[qi + 1]])
        assert len(got) == min(int(ks[qi]), n)
        outside = [o for o in range(n) if o not in got]
        assert max(ex[s] for s in got) <= min(ex[o] for o in outside)
        assert got == sorted(range(n), key=lambda o: (ex[o], o))[:len(got)]


def test_range_and_knn_strings_by_exhaustion():
    rng = np.random.default_rng(12)
    items = [bytes(rng.choice(list(b"ab"), size=int(rng.integers(0, 6))).tolist()) for _ in range(150)]
    S = strings_from_list(items)
    qitems = [bytes(rng.choice(list(b"ab"), size=int(rng.integers(0, 6))).tolist()) for _ in range(15)]
    Qs = strings_from_list(qitems)
    radii = rng.integers(0, 4, size=15).astype(np.float32) + 0.5   # edit radii are floored
    ks = rng.integers(1, 20, size=15).astype(np.int32)
    off, ids, dist, _ = oracle.range_query("edit", S, Qs, radii)
    koff, kids, kdist, _ = oracle.knn_query("edit", S, Qs, ks)
    for qi, q in enumerate(qitems):
        bfs = _bfs_distances(q.decode(), "ab", 6)
        ex = [bfs[s.decode()] for s in items]
        want = [o for o in range(150) if ex[o] <= int(radii[qi])]
        assert list(ids[off[qi]:off[qi + 1]]) == want
        assert list(dist[off[qi]:off[qi + 1]]) == [ex[o] for o in want]
        got = list(kids[koff[qi]:koff[qi + 1]])
        assert got == sorted(range(150), key=lambda o: (ex[o], o))[:int(ks[qi])]


def test_visibility_by_sequence_numbers():
    """Stream updates (Section 4.4): the answer at sequence s is the brute-force
    answer over the objects inserted before s and not deleted before s."""
    rng = np.random.default_rng(13)
    n, D = 300, 4
    X = rng.standard_normal((n, D)).astype(np.float32)
    ins = np.full(n, -1, np.int64)
    ins[200:] = np.arange(100) * 3 + 1                      # inserted during the stream
    dele = np.full(n, np.iinfo(np.int64).max, np.int64)
    victims = rng.choice(n, size=60, replace=False)
    dele[victims] = rng.integers(0, 320, size=60)
    dele = np.maximum(dele, np.where(dele < np.iinfo(np.int64).max, ins + 1, dele))
    Q = rng.standard_normal((25, D)).astype(np.float32)
    qseq = rng.integers(0, 330, size=25) * 2              # even: no clash with odd insert seqs
    radii = np.full(25, 1.5, np.float32)
    off, ids, _, _ = oracle.range_query("l2", X, Q, radii, ins, dele, qseq)
    koff, kids, _, _ = oracle.knn_query("l2", X, Q, 7, ins, dele, qseq)
    for qi in range(25):
        s = qseq[qi]
        live = [o for o in range(n) if ins[o] < s and not (dele[o] <= s)]
        sub = X[live]
        o2, i2, _, _ = oracle.range_query("l2", sub, Q[qi:qi + 1], radii[qi:qi + 1])
        assert list(ids[off[qi]:off[qi + 1]]) == [live[j] for j in i2]
        o3, i3, _, _ = oracle.knn_query("l2", sub, Q[qi:qi + 1], 7)
        assert list(kids[koff[qi]:koff[qi + 1]]) == [live[j] for j in i3]


# ------------------------------------------------------------ index construction

def _check_index(objects, metric, T):
    n, F, h = T["n"], T["fanout"], T["h"]
    perm, table = T["perm"], T["table"]
    assert sorted(perm.tolist()) == list(range(n))                  # leaves partition the set
    assert sum(F ** i for i in range(h + 1)) == sum(len(s) for s in T["size"])
    for l in range(h + 1):
        for i in range(F ** l):
            s, c = T["pos"][l][i], T["size"][l][i]
            if l > 0:
                ps, pc = T["pos"][l - 1][i // F], T["size"][l - 1][i // F]
                j = i % F
                avg = pc // F
                assert c == (avg if j < F - 1 else pc - avg * (F - 1))   # even split, remainder last
                assert s == ps + j * avg
                if c:
                    col = table[l - 1, s:s + c]
                    assert T["lo"][l][i] == col.min() and T["hi"][l][i] == col.max()
                    # siblings were cut from one run sorted by (distance, id): intervals in
                    # order, and where the cut falls inside a run of tied distances the
                    # earlier child holds the smaller ids
                    if j > 0 and T["size"][l][i - 1]:
                        assert T["hi"][l][i - 1] <= T["lo"][l][i]
                        if T["hi"][l][i - 1] == T["lo"][l][i]:
                            ps0, pc0 = T["pos"][l][i - 1], T["size"][l][i - 1]
                            prev = perm[ps0:ps0 + pc0][table[l - 1, ps0:ps0 + pc0] == T["lo"][l][i]]
                            cur = perm[s:s + c][col == T["lo"][l][i]]
                            assert prev.max() < cur.min()
                    # the ancestor pivot's distance, recomputed from scratch
                    p = T["pivot"][l - 1][i // F]
                    objs = objects.take(perm[s:s + c]) if isinstance(objects, Strings) else objects[perm[s:s + c]]
                    tgt = objects.get(int(p)) if isinstance(objects, Strings) else objects[p]
                    assert np.array_equal(oracle.distances_to(metric, objs, tgt).astype(np.float32), col)
            if l < h and c:
                p = T["pivot"][l][i]
                assert p in set(perm[s:s + c].tolist())                  # the pivot is one of the node's objects
                if l > 0:
                    # farthest-first: no object of the node is farther from the ancestor pivots
                    sc = table[:l, s:s + c].min(axis=0)
                    prow = int(np.nonzero(perm[s:s + c] == p)[0][0])
                    assert sc[prow] == sc.max()
                    assert p == perm[s:s + c][sc == sc.max()].min()


def _check_leaf_order(T):
    """Rows of a leaf come in the order of the last sort: (distance to the
    leaf's parent pivot, id) ascending."""
    h, F = T["h"], T["fanout"]
    for i in range(F ** h):
        s, c = T["pos"][h][i], T["size"][h][i]
        d, ids = T["table"][h - 1, s:s + c], T["perm"][s:s + c]
        for a in range(c - 1):
            assert d[a] < d[a + 1] or (d[a] == d[a + 1] and ids[a] < ids[a + 1])


def test_index_oracle_tie_order_by_hand():
    """Every object at the same L1 distance 2 from the root pivot (object 0,
    the origin): Algorithm 3 sorts the node by (distance, id), so the pivot
    (distance 0) comes first, the tied objects follow in ascending id, and the
    even split of 41 objects into 4 children of 10 (the last takes 11) cuts
    that order into consecutive id ranges -- the whole tree is known by hand."""
    rng = np.random.default_rng(23)
    X = np.zeros((41, 6), np.float32)
    for o in range(1, 41):
        a, b = rng.choice(6, 2, replace=False)      # two coordinates of 1: |x|_1 = 2 exactly
        X[o, a] = X[o, b] = 1.0
    T = build_index(X, "l1", 4, 1, root_pivot=0)
    assert T["h"] == 1
    assert T["perm"].tolist() == list(range(41))
    assert T["size"][1].tolist() == [10, 10, 10, 11] and T["pos"][1].tolist() == [0, 10, 20, 30]
    assert T["lo"][1].tolist() == [0.0, 2.0, 2.0, 2.0] and T["hi"][1].tolist() == [2.0, 2.0, 2.0, 2.0]
    assert T["table"][0].tolist() == [0.0] + [2.0] * 40
    _check_index(X, "l1", T)
    _check_leaf_order(T)
    # reversed ids: the same points listed backwards keep the pivot first and
    # the tied ones in ascending id again
    Xr = np.concatenate([X[:1], X[1:][::-1]])
    Tr = build_index(Xr, "l1", 4, 1, root_pivot=0)
    assert Tr["perm"].tolist() == list(range(41))


def test_index_oracle_vectors():
    rng = np.random.default_rng(21)
    X = (rng.standard_normal((700, 5))).astype(np.float32)
    X[600:] = X[:100]                                              # duplicates
    T = build_index(X, "l2", 4, 0, root_pivot=17)
    assert T["h"] == height(700, 4) == 4
    _check_index(X, "l2", T)
    _check_leaf_order(T)
    T1 = build_index(X, "l1", 6, 2, root_pivot=3)
    _check_index(X, "l1", T1)
    _check_leaf_order(T1)
    # integer points: many exactly tied distances at every level
    Xi = rng.integers(0, 3, size=(500, 3)).astype(np.float32)
    T2 = build_index(Xi, "l1", 5, 3, root_pivot=11)
    _check_index(Xi, "l1", T2)
    _check_leaf_order(T2)


def test_index_oracle_strings():
    rng = np.random.default_rng(22)
    items = [bytes(rng.choice(list(b"abcd"), size=int(rng.integers(1, 9))).tolist()) for _ in range(400)]
    S = strings_from_list(items)
    T = build_index(S, "edit", 5, 3, root_pivot=0)
    _check_index(S, "edit", T)
    _check_leaf_order(T)


def test_height_formula():
    # Algorithm 1: h = ceil(log_Nc(|O| + 1)) - 1 (at least one pivot level)
    assert height(10_000, 8, 5) == 5
    assert height(1_000_000, 20) == 4
    assert height(10_000_000, 20) == 5
    assert height(2_000_000, 20) == 4
    assert height(399, 20) == 1 and height(400, 20) == 2
    assert height(1, 20) == 1
