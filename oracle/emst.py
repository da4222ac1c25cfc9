"""Float64 reference of the Euclidean minimum spanning tree -- TEST
INFRASTRUCTURE ONLY.

Only the tests and ``bench.py``'s CPU legs import this module; the CUDA
library never calls it.

Problem (Section 7, "Boruvka's Algorithm"): the minimum spanning tree of the
complete graph on S_r with Euclidean edge weights.  Readings:

* an edge's weight is compared through its float64 squared length (the sum of
  (p_j - q_j)^2 over j, left to right, from the float32 inputs); it is
  reported as the correctly rounded square root;
* edges of equal weight are ordered by (lower endpoint index, higher endpoint
  index), so every edge has its own rank and the tree is unique: the
  minimum spanning tree under the order (d^2, min index, max index);
* each edge is reported as (lower index, higher index).

``emst_kruskal`` is that definition written out (Kruskal's algorithm over all
pairs, sorted by the order).  ``emst_prim`` grows the tree from point 0,
always adding the smallest crossing edge under the same order: an
independent algorithm for the same unique tree, used to pin the first.
Both are O(n^2) in memory or time: small inputs only.
"""
from __future__ import annotations

from typing import Tuple

import numpy as np

from .kfn import _d2_rows


def _pairs(P: np.ndarray):
    X = np.asarray(P, dtype=np.float32).astype(np.float64)
    n = X.shape[0]
    D = _d2_rows(X, X)
    iu, ju = np.triu_indices(n, k=1)
    return n, D, iu.astype(np.int64), ju.astype(np.int64)


def emst_kruskal(P: np.ndarray) -> Tuple[np.ndarray, np.ndarray]:
    """(edges int64 (n - 1, 2) as (lo, hi), d2 float64 (n - 1)) in the order
    Kruskal's algorithm adds them (ascending under the edge order)."""
    n, D, iu, ju = _pairs(P)
    w = D[iu, ju]
    order = np.lexsort((ju, iu, w))
    parent = np.arange(n)

    def find(a):
        while parent[a] != a:
            parent[a] = parent[parent[a]]
            a = parent[a]
        return a

    edges, wts = [], []
    for e in order:
        a, b = find(iu[e]), find(ju[e])
        if a != b:
            parent[max(a, b)] = min(a, b)
            edges.append((iu[e], ju[e]))
            wts.append(w[e])
            if len(edges) == n - 1:
                break
    return np.array(edges, dtype=np.int64).reshape(-1, 2), np.array(wts, dtype=np.float64)


def emst_prim(P: np.ndarray) -> Tuple[np.ndarray, np.ndarray]:
    """The same tree grown from point 0 (edges in the order Prim adds them)."""
    X = np.asarray(P, dtype=np.float32).astype(np.float64)
    n = X.shape[0]
    inside = np.zeros(n, dtype=bool)
    inside[0] = True
    # each outside point's best crossing edge: (d2, lo, hi) and its tree end
    bd = _d2_rows(X[:1], X)[0]
    blo = np.minimum(0, np.arange(n))
    bhi = np.maximum(0, np.arange(n))
    edges, wts = [], []
    for _ in range(n - 1):
        out = np.nonzero(~inside)[0]
        o = np.lexsort((bhi[out], blo[out], bd[out]))[0]
        v = out[o]
        edges.append((blo[v], bhi[v]))
        wts.append(bd[v])
        inside[v] = True
        d = _d2_rows(X[v:v + 1], X)[0]
        lo, hi = np.minimum(v, np.arange(n)), np.maximum(v, np.arange(n))
        better = (~inside) & ((d < bd) | ((d == bd) & ((lo < blo) | ((lo == blo) & (hi < bhi)))))
        bd[better], blo[better], bhi[better] = d[better], lo[better], hi[better]
    return np.array(edges, dtype=np.int64).reshape(-1, 2), np.array(wts, dtype=np.float64)


def canonical(edges: np.ndarray, d2: np.ndarray) -> Tuple[np.ndarray, np.ndarray]:
    """Edges sorted by (lo, hi), for comparing edge sets."""
    e = np.asarray(edges, dtype=np.int64).reshape(-1, 2)
    order = np.lexsort((e[:, 1], e[:, 0]))
    return e[order], np.asarray(d2)[order]
