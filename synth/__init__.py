"""Seeded synthetic inputs for GTS range / kNN search.

This module only draws random numbers and lays them out; it holds none of the
search method's arithmetic (no distances, no pruning, no selection).  Both the
CPU oracle (tests) and the CUDA library path consume the same arrays.

The paper's datasets (Words, DNA, T-Loc, Color; Section 6.1, Table 2) are not
available, so these generators stand in for them with the shapes listed below.
All randomness comes from numpy's PCG64 with the seed stated per workload.

Layouts
-------
* vectors: float32, row-major ``[n, dim]``.
* strings: CSR ``(data uint8[total], offsets int64[n + 1])``; string ``i`` is
  ``data[offsets[i]:offsets[i + 1]]``.
"""
from __future__ import annotations

import dataclasses
import os
from typing import Optional

import numpy as np

LOWER = np.frombuffer(b"abcdefghijklmnopqrstuvwxyz", dtype=np.uint8)
ACGT = np.frombuffer(b"ACGT", dtype=np.uint8)


@dataclasses.dataclass
class Strings:
    data: np.ndarray      # uint8[total]
    offsets: np.ndarray   # int64[n + 1]

    @property
    def n(self) -> int:
        return int(self.offsets.shape[0] - 1)

    def get(self, i: int) -> bytes:
        return bytes(self.data[self.offsets[i]:self.offsets[i + 1]])

    def lengths(self) -> np.ndarray:
        return np.diff(self.offsets)

    def take(self, idx) -> "Strings":
        return strings_from_list([self.get(int(i)) for i in idx])


def strings_from_list(items) -> Strings:
    lens = np.fromiter((len(s) for s in items), dtype=np.int64, count=len(items))
    offsets = np.zeros(len(items) + 1, dtype=np.int64)
    np.cumsum(lens, out=offsets[1:])
    data = np.frombuffer(b"".join(items), dtype=np.uint8).copy() if len(items) else np.zeros(0, np.uint8)
    return Strings(data, offsets)


@dataclasses.dataclass
class Workload:
    """One synthetic workload: objects, queries and the query parameters."""
    name: str
    metric: str                      # "edit" | "l1" | "l2" | "cos"
    objects: object                  # np.ndarray [n, dim] float32, or Strings
    queries: object                  # same kind as objects
    kind: str                        # "range" | "knn" | "mixed"
    radii: Optional[np.ndarray] = None   # float32[nq] (range)
    k: Optional[np.ndarray] = None       # int32[nq] (knn)
    fanout: int = 20
    n_pivots: int = 0                # 0 = height from the node capacity (Algorithm 1)
    extra: dict = dataclasses.field(default_factory=dict)

    @property
    def n(self) -> int:
        return self.objects.n if isinstance(self.objects, Strings) else int(self.objects.shape[0])

    @property
    def nq(self) -> int:
        return self.queries.n if isinstance(self.queries, Strings) else int(self.queries.shape[0])


# ---------------------------------------------------------------------------
# strings
# ---------------------------------------------------------------------------

def random_strings(n: int, lmin: int, lmax: int, alphabet: np.ndarray, rng) -> Strings:
    lens = rng.integers(lmin, lmax + 1, size=n).astype(np.int64)
    offsets = np.zeros(n + 1, dtype=np.int64)
    np.cumsum(lens, out=offsets[1:])
    data = alphabet[rng.integers(0, alphabet.shape[0], size=int(offsets[-1]))]
    return Strings(data.astype(np.uint8), offsets)


def mutate(s: bytes, n_edits: int, alphabet: np.ndarray, rng) -> bytes:
    """Apply ``n_edits`` random unit edits (substitute / insert / delete, each
    with probability 1/3; uniform position and letter).  A delete that would
    empty the string becomes a substitution, so the length stays >= 1."""
    b = bytearray(s)
    for _ in range(n_edits):
        op = int(rng.integers(0, 3))
        if op == 2 and len(b) <= 1:
            op = 0
        if op == 0 and len(b) == 0:
            op = 1
        if op == 0:
            b[int(rng.integers(0, len(b)))] = int(alphabet[int(rng.integers(0, alphabet.shape[0]))])
        elif op == 1:
            b.insert(int(rng.integers(0, len(b) + 1)), int(alphabet[int(rng.integers(0, alphabet.shape[0]))]))
        else:
            del b[int(rng.integers(0, len(b)))]
    return bytes(b)


def words_like(n: int = 10_000, nq: int = 256, radius: float = 2.0, seed: int = 0,
               qseed: int = 1, fanout: int = 8, n_pivots: int = 5) -> Workload:
    """Lower-case strings, length uniform in 4..16; queries are dataset strings
    with 0..3 random edits.  Edit distance, range queries of radius 2, 5 pivot
    levels, node capacity 8.  Stands in for the Words dataset (Table 2)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    objs = random_strings(n, 4, 16, LOWER, rng)
    qrng = np.random.Generator(np.random.PCG64(qseed))
    picks = qrng.integers(0, n, size=nq)
    qs = []
    for i in picks:
        ne = int(qrng.integers(0, 4))
        qs.append(mutate(objs.get(int(i)), ne, LOWER, qrng))
    queries = strings_from_list(qs)
    return Workload("words_10k_r2", "edit", objs, queries, "range",
                    radii=np.full(nq, radius, np.float32), fanout=fanout, n_pivots=n_pivots)


def dna_like(n_seeds: int = 10_000, copies: int = 100, length: int = 108, nq: int = 20_000,
             radius: float = 8.0, seed: int = 0, qseed: int = 1, fanout: int = 20,
             n_pivots: int = 0) -> Workload:
    """DNA strings: ``n_seeds`` random ACGT seeds of ``length``; each seed gives
    ``copies`` strings with 1..6 random edits (the seeds themselves are not in
    the set).  Queries: a uniform seed with 1..6 edits.  Edit distance, range
    radius 8.  Stands in for the DNA dataset (1M x 108, Table 2)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    seeds = random_strings(n_seeds, length, length, ACGT, rng)
    seed_list = [seeds.get(i) for i in range(n_seeds)]
    items = []
    for i in range(n_seeds):
        s = seed_list[i]
        for _ in range(copies):
            items.append(mutate(s, int(rng.integers(1, 7)), ACGT, rng))
    objs = strings_from_list(items)
    qrng = np.random.Generator(np.random.PCG64(qseed))
    qs = [mutate(seed_list[int(qrng.integers(0, n_seeds))], int(qrng.integers(1, 7)), ACGT, qrng)
          for _ in range(nq)]
    return Workload(f"dna_{n_seeds * copies}_r{int(radius)}", "edit", objs, strings_from_list(qs),
                    "range", radii=np.full(nq, radius, np.float32), fanout=fanout, n_pivots=n_pivots)


# ---------------------------------------------------------------------------
# vectors
# ---------------------------------------------------------------------------

def gaussian_mixture(n: int = 1_000_000, dim: int = 128, n_centers: int = 64, sigma: float = 0.1,
                     nq: int = 10_000, k: int = 10, seed: int = 0, qseed: int = 1,
                     fanout: int = 20) -> Workload:
    """``n`` float32 vectors from ``n_centers`` equally weighted isotropic
    Gaussians (centres uniform in [-1, 1]^dim, standard deviation ``sigma``).
    Queries come from the same mixture with ``qseed``.  L2 kNN with ``k``."""
    rng = np.random.Generator(np.random.PCG64(seed))
    centers = rng.uniform(-1.0, 1.0, size=(n_centers, dim))
    lab = rng.integers(0, n_centers, size=n)
    X = np.empty((n, dim), dtype=np.float32)
    step = 1 << 18
    for s in range(0, n, step):
        e = min(n, s + step)
        X[s:e] = (centers[lab[s:e]] + sigma * rng.standard_normal((e - s, dim))).astype(np.float32)
    qrng = np.random.Generator(np.random.PCG64(qseed))
    qlab = qrng.integers(0, n_centers, size=nq)
    Q = (centers[qlab] + sigma * qrng.standard_normal((nq, dim))).astype(np.float32)
    return Workload(f"gauss{n_centers}_{n}x{dim}_knn{k}", "l2", X, Q, "knn",
                    k=np.full(nq, k, np.int32), fanout=fanout)


def zipf_clusters_2d(n: int = 10_000_000, n_clusters: int = 1000, zipf_s: float = 1.1,
                     sigma: float = 0.01, nq: int = 100_000, seed: int = 0, qseed: int = 1,
                     fanout: int = 20, radius: Optional[float] = None) -> Workload:
    """2-D points from ``n_clusters`` Gaussian clusters whose weights fall as
    rank^-zipf_s; centres uniform in [0,1]^2, standard deviation ``sigma``.
    Range queries from the same distribution.  Stands in for T-Loc (10M x 2).
    ``radius`` is left to the caller to calibrate (about 0.01% selectivity)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    centers = rng.uniform(0.0, 1.0, size=(n_clusters, 2))
    w = np.arange(1, n_clusters + 1, dtype=np.float64) ** (-zipf_s)
    w /= w.sum()
    lab = rng.choice(n_clusters, size=n, p=w)
    X = (centers[lab] + sigma * rng.standard_normal((n, 2))).astype(np.float32)
    qrng = np.random.Generator(np.random.PCG64(qseed))
    qlab = qrng.choice(n_clusters, size=nq, p=w)
    Q = (centers[qlab] + sigma * qrng.standard_normal((nq, 2))).astype(np.float32)
    wl = Workload(f"zipf2d_{n}", "l2", X, Q, "range", fanout=fanout)
    wl.extra["centers"] = centers
    wl.extra["weights"] = w
    if radius is not None:
        wl.radii = np.full(nq, radius, np.float32)
    return wl


def zipf_points(centers: np.ndarray, weights: np.ndarray, sigma: float, m: int, seed: int) -> np.ndarray:
    """More points from the same cluster mixture (used for streamed inserts)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    lab = rng.choice(centers.shape[0], size=m, p=weights)
    return (centers[lab] + sigma * rng.standard_normal((m, 2))).astype(np.float32)


def uniform_cube(n: int = 2_000_000, dim: int = 256, nq: int = 20_000, seed: int = 0,
                 qseed: int = 1, fanout: int = 20) -> Workload:
    """``n`` float32 vectors uniform in [0,1]^dim and ``nq`` queries from the
    same law.  L1 metric.  Stands in for Color (Table 2)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    X = np.empty((n, dim), dtype=np.float32)
    step = 1 << 18
    for s in range(0, n, step):
        e = min(n, s + step)
        X[s:e] = rng.random((e - s, dim), dtype=np.float32)
    qrng = np.random.Generator(np.random.PCG64(qseed))
    Q = qrng.random((nq, dim), dtype=np.float32)
    return Workload(f"uniform_{n}x{dim}_l1", "l1", X, Q, "mixed", fanout=fanout)


def word_vectors(n: int = 200_000, dim: int = 300, n_centers: int = 500, nq: int = 10_000, k: int = 10,
                 seed: int = 0, qseed: int = 1, fanout: int = 20) -> Workload:
    """``n`` float32 vectors shaped like word embeddings: a shared mean
    direction, ``n_centers`` topic clusters, and per-coordinate scales that
    fall as (j + 1)^-0.3 (an anisotropic spectrum); ``nq`` queries from the
    same law.  Angular (cosine) kNN with ``k``.  Stands in for Vector (Table
    2: 200K x 300, cosine)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    scale = (np.arange(dim) + 1.0) ** -0.3
    mean = 0.5 * rng.standard_normal(dim) * scale
    centers = rng.standard_normal((n_centers, dim)) * scale
    lab = rng.integers(0, n_centers, size=n)
    X = np.empty((n, dim), dtype=np.float32)
    step = 1 << 16
    for s in range(0, n, step):
        e = min(n, s + step)
        X[s:e] = (mean + centers[lab[s:e]] + 0.6 * rng.standard_normal((e - s, dim)) * scale).astype(np.float32)
    qrng = np.random.Generator(np.random.PCG64(qseed))
    qlab = qrng.integers(0, n_centers, size=nq)
    Q = (mean + centers[qlab] + 0.6 * qrng.standard_normal((nq, dim)) * scale).astype(np.float32)
    return Workload(f"wordvec_{n}x{dim}_cos_knn{k}", "cos", X, Q, "knn", k=np.full(nq, k, np.int32), fanout=fanout)


@dataclasses.dataclass
class MultiWorkload:
    """Several columns of one object set, one index per column: row i of
    every column describes object i."""
    name: str
    metrics: list                    # per column "l1" | "l2" | "cos"
    objects: list                    # per column np.ndarray [n, dim_j] float32
    queries: list                    # per column np.ndarray [nq, dim_j] float32
    k: np.ndarray                    # int32[nq]
    fanout: int = 20


def multi_columns(n: int = 200_000, nq: int = 10_000, k: int = 10, n_centers: int = 500, latent: int = 16,
                  seed: int = 0, qseed: int = 1, fanout: int = 20) -> MultiWorkload:
    """Two columns of ``n`` objects, like items with an image embedding (L2,
    128 dimensions) and a text embedding (angle, 300 dimensions, the word
    vectors' anisotropic law): both columns of an object derive from its
    topic (one of ``n_centers``) and a ``latent``-dimensional offset of its
    own through a fixed linear map per column, plus independent column noise.
    The L2 column is scaled so that its distances are of the order of the
    angles (about 1), so both columns weigh in the sum.  ``nq`` queries from
    the same law; kNN with ``k``."""
    rng = np.random.Generator(np.random.PCG64(seed))
    C0 = rng.standard_normal((n_centers, 128))
    W0 = 0.25 * rng.standard_normal((latent, 128))
    scale = (np.arange(300) + 1.0) ** -0.3
    mean = 0.5 * rng.standard_normal(300) * scale
    C1 = rng.standard_normal((n_centers, 300)) * scale
    W1 = 0.25 * rng.standard_normal((latent, 300)) * scale

    def draw(r, m):
        X0 = np.empty((m, 128), np.float32)
        X1 = np.empty((m, 300), np.float32)
        step = 1 << 16
        for s in range(0, m, step):
            e = min(m, s + step)
            lab = r.integers(0, n_centers, size=e - s)
            z = r.standard_normal((e - s, latent))
            X0[s:e] = 0.07 * (C0[lab] + z @ W0 + 0.5 * r.standard_normal((e - s, 128)))
            X1[s:e] = mean + C1[lab] + z @ W1 + 0.5 * r.standard_normal((e - s, 300)) * scale
        return X0, X1

    X0, X1 = draw(rng, n)
    Q0, Q1 = draw(np.random.Generator(np.random.PCG64(qseed)), nq)
    return MultiWorkload(f"multicol_{n}_l2x128_cos300_knn{k}", ["l2", "cos"], [X0, X1], [Q0, Q1],
                         np.full(nq, k, np.int32), fanout=fanout)


def poisson_arrivals(m: int, rate_qps: float, seed: int) -> np.ndarray:
    """Open-loop arrival times (seconds from 0) of ``m`` requests at mean rate
    ``rate_qps``."""
    rng = np.random.Generator(np.random.PCG64(seed))
    return np.cumsum(rng.exponential(1.0 / rate_qps, size=m))


def mixed_requests(nq: int, seed: int, kmax: int = 100):
    """For the serving mix: a boolean ``is_knn`` per request (50/50) and a k in
    1..kmax for the kNN ones."""
    rng = np.random.Generator(np.random.PCG64(seed))
    is_knn = rng.random(nq) < 0.5
    k = rng.integers(1, kmax + 1, size=nq).astype(np.int32)
    return is_knn, k


def update_stream(n_queries: int, n_inserts: int, n_deletes: int, seed: int) -> np.ndarray:
    """An interleaving of operation kinds: 0 = query, 1 = insert, 2 = delete,
    uniformly shuffled with ``seed``."""
    ops = np.concatenate([np.zeros(n_queries, np.int8), np.ones(n_inserts, np.int8),
                          np.full(n_deletes, 2, np.int8)])
    rng = np.random.Generator(np.random.PCG64(seed))
    rng.shuffle(ops)
    return ops


def random_choice(n: int, m: int, seed: int) -> np.ndarray:
    rng = np.random.Generator(np.random.PCG64(seed))
    return rng.integers(0, n, size=m)


def small_vectors(n: int, dim: int, nq: int, seed: int, kind: str = "gauss", dup_frac: float = 0.0):
    """Small seeded vector sets for parity tests.  ``dup_frac`` of the objects
    are exact copies of other objects (the duplicate-heavy case)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    if kind == "gauss":
        centers = rng.uniform(-1, 1, size=(max(1, n // 200), dim))
        lab = rng.integers(0, centers.shape[0], size=n)
        X = (centers[lab] + 0.1 * rng.standard_normal((n, dim))).astype(np.float32)
        ql = rng.integers(0, centers.shape[0], size=nq)
        Q = (centers[ql] + 0.1 * rng.standard_normal((nq, dim))).astype(np.float32)
    else:
        X = rng.random((n, dim), dtype=np.float32)
        Q = rng.random((nq, dim), dtype=np.float32)
    if dup_frac > 0 and n > 1:
        m = int(n * dup_frac)
        dst = rng.choice(n, size=m, replace=False)
        src = rng.integers(0, n, size=m)
        X[dst] = X[src]
    return X, Q


def cache_dir() -> str:
    d = os.environ.get("GTS_SYNTH_CACHE", os.path.join("/tmp", "gts_synth_cache"))
    os.makedirs(d, exist_ok=True)
    return d
