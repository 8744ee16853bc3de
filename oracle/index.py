"""Index construction of GTS (Section 4.3, Algorithms 1-3), step by step in
numpy -- TEST INFRASTRUCTURE ONLY (see the package docstring).

Readings of the paper used here (each one is also listed in the design notes):

* Height (Algorithm 1, first step): h = ceil(log_Nc(|O| + 1)) - 1, at least 1,
  unless the caller fixes the number of pivot levels.
* Node numbering (Section 4.2, Eq. 1): level by level; child j of the node with
  0-based index i at one level is node i * Nc + j of the next level.
* Pivot choice (Algorithm 2, FFT): the root pivot is a caller-given random
  object; at deeper levels a node's pivot is the object of the node whose
  smallest distance to the pivots already chosen on its path (its ancestors)
  is largest, ties to the smallest object id.  An empty node has no pivot.
* Mapping (Algorithm 2): every object of a node gets its distance to the
  node's pivot, computed exactly (FP64 / integer) and stored as float32.
* Partitioning (Algorithm 3): the objects of every node are sorted by
  (distance to the node's pivot, object id) -- the paper's encoded key
  i + dis/(max+1) orders by node first, then distance; the id breaks ties so
  the tree is unique -- then split by count into Nc children of
  floor(size/Nc) objects each, the last child taking the remainder.
* Child bounds: the paper keeps min_dis (the child's first distance to the
  parent pivot); this index also keeps the last one (max), so a child holds
  the interval [lo, hi] of its objects' distances to the parent pivot.  An
  empty child has lo = +inf, hi = -inf.
* Table list (Section 4.2): one row per object in final (leaf) order, with
  the distance to the pivot of each of its h ancestors (all h columns).
"""
from __future__ import annotations

import numpy as np

from synth import Strings
from . import distances_to


def height(n: int, fanout: int, n_pivots: int = 0) -> int:
    if n_pivots > 0:
        return int(n_pivots)
    # smallest t with fanout**t >= n + 1, i.e. ceil(log_fanout(n + 1)), in integers
    t, p = 0, 1
    while p < n + 1:
        p *= fanout
        t += 1
    return max(1, t - 1)


def _object(objects, i):
    if isinstance(objects, Strings):
        return objects.get(int(i))
    return objects[int(i)]


def _subset(objects, idx):
    if isinstance(objects, Strings):
        return objects.take(idx)
    return objects[idx]


def build_index(objects, metric: str, fanout: int, n_pivots: int, root_pivot: int) -> dict:
    """Returns the whole tree:

    ``h``, ``fanout``; ``perm`` int64[n] (row -> object id, leaf order);
    ``table`` float32[h, n] (row's distance to its level-l ancestor's pivot);
    per level l = 0..h: ``pos[l]``, ``size[l]`` (int64[Nc**l]) and for l >= 1
    ``lo[l]``, ``hi[l]`` (float32[Nc**l]); per pivot level l = 0..h-1
    ``pivot[l]`` (int64[Nc**l], object id or -1).
    """
    n = objects.n if isinstance(objects, Strings) else int(objects.shape[0])
    F = int(fanout)
    h = height(n, F, n_pivots)
    perm = np.arange(n, dtype=np.int64)
    table = np.zeros((h, n), np.float32)
    pos = [np.zeros(1, np.int64)]
    size = [np.array([n], np.int64)]
    lo = [None]
    hi = [None]
    pivots = []
    for l in range(h):
        nn = F ** l
        piv = np.full(nn, -1, np.int64)
        # ---- Mapping (Algorithm 2) ----
        for i in range(nn):
            s, c = int(pos[l][i]), int(size[l][i])
            if c == 0:
                continue
            rows = perm[s:s + c]
            if l == 0:
                p = int(root_pivot)
            else:
                score = table[:l, s:s + c].min(axis=0)          # distance to the nearest ancestor pivot
                best = score.max()
                p = int(rows[score == best].min())              # farthest-first; ties -> smallest id
            piv[i] = p
            d = distances_to(metric, _subset(objects, rows), _object(objects, p))
            table[l, s:s + c] = d.astype(np.float32)
        pivots.append(piv)
        # ---- Partitioning (Algorithm 3) ----
        npos = np.zeros(nn * F, np.int64)
        nsize = np.zeros(nn * F, np.int64)
        nlo = np.full(nn * F, np.inf, np.float32)
        nhi = np.full(nn * F, -np.inf, np.float32)
        for i in range(nn):
            s, c = int(pos[l][i]), int(size[l][i])
            if c > 0:
                order = np.lexsort((perm[s:s + c], table[l, s:s + c]))   # by distance, then id
                perm[s:s + c] = perm[s:s + c][order]
                table[:l + 1, s:s + c] = table[:l + 1, s:s + c][:, order]
            avg = c // F
            for j in range(F):
                cs = s + j * avg
                cc = avg if j < F - 1 else c - avg * (F - 1)
                npos[i * F + j] = cs
                nsize[i * F + j] = cc
                if cc > 0:
                    nlo[i * F + j] = table[l, cs]
                    nhi[i * F + j] = table[l, cs + cc - 1]
        pos.append(npos)
        size.append(nsize)
        lo.append(nlo)
        hi.append(nhi)
    return dict(h=h, fanout=F, n=n, perm=perm, table=table, pos=pos, size=size, lo=lo, hi=hi,
                pivot=pivots)
