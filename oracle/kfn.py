"""Float64 reference of k-furthest-neighbour search -- TEST INFRASTRUCTURE ONLY.

Only the tests and ``bench.py``'s CPU legs (its ``cpu_baseline`` and
reference arm) import this module; the CUDA library never calls it.

Problem (Section 5, the paragraph on k-furthest neighbour search after
Algorithm 4): for every query, the k reference points at the LARGEST
Euclidean distance, with the kNN rules inverted -- lists sorted by descending
distance, distances initialised to 0, and a candidate kept when d > D[k].
Readings shared with the kNN oracle:

* ties are broken by the lower reference index, so the result is unique: the
  first k of the list sorted by (distance descending, index ascending);
* a monochromatic query never returns itself (by index);
* squared distances are float64 sums of (q_j - r_j)^2 over j left to right,
  one rounding per operation, from the float32 inputs.

``kfn_brute`` is that definition written out.  ``kfn_dualtree`` is the
meta-algorithm of Section 2 (Algorithm 1's depth-first traversal) with the
inverted Score and BaseCase, on kd-trees, kept only as an independent check of
the definition on small inputs (pure Python loops).  Its bound is the
inversion of the sound kNN bound: for a query node N,

    B1'(N) = min over descendant points p of D_p[k],
    A'(N)  = max over descendant points p of D_p[k],
    B'(N)  = max over N and its ancestors a of max(B1'(a), A'(a) - 2 lambda(a)),

where D_p[k] is p's current k-th furthest distance (0 while p has fewer than k
candidates) and lambda the largest distance from a node's box centre to its
points.  A'(a) - 2 lambda(a) holds for every point of a by the triangle
inequality (two points of a are at most 2 lambda apart).  A pair is pruned
when d_max(N_q, N_r) < B'(N_q), strictly, so that an equal-distance,
lower-index point is never lost.
"""
from __future__ import annotations

from typing import Optional, Tuple

import numpy as np


def _d2_rows(Q: np.ndarray, R: np.ndarray) -> np.ndarray:
    """(len(Q), len(R)) float64 squared distances, summed left to right."""
    s = np.zeros((Q.shape[0], R.shape[0]), dtype=np.float64)
    for j in range(Q.shape[1]):
        t = Q[:, j:j + 1] - R[None, :, j]
        s = s + t * t
    return s


def kfn_brute(ref: np.ndarray, query: Optional[np.ndarray], k: int,
              self_idx: Optional[np.ndarray] = None,
              chunk: int = 256) -> Tuple[np.ndarray, np.ndarray]:
    """Exact k-furthest neighbours by comparing every pair (the definition).

    ``query is None`` means monochromatic (query i never returns reference i);
    ``self_idx`` names the reference each query must skip (-1 for none).
    Returns (idx int64 (n, k), d2 float64 (n, k)), descending by squared
    distance, ties by ascending index.
    """
    R = np.asarray(ref, dtype=np.float32).astype(np.float64)
    if query is None:
        Q = R
        self_idx = np.arange(R.shape[0], dtype=np.int64)
    else:
        Q = np.asarray(query, dtype=np.float32).astype(np.float64)
    m, n = R.shape[0], Q.shape[0]
    avail = m - (0 if self_idx is None else 1)
    if not 0 < k <= avail:
        raise ValueError("k out of range")
    out_i = np.empty((n, k), dtype=np.int64)
    out_d = np.empty((n, k), dtype=np.float64)
    for c0 in range(0, n, chunk):
        D = _d2_rows(Q[c0:c0 + chunk], R)
        rows = np.arange(D.shape[0])
        if self_idx is not None:
            s = np.asarray(self_idx[c0:c0 + chunk], dtype=np.int64)
            keep = s >= 0
            D[rows[keep], s[keep]] = -np.inf  # never selected: k <= m - 1
        # the k-th largest value of each row; every point at or above it is a
        # candidate (ties included), ranked by (distance desc, index asc)
        thr = -np.partition(-D, k - 1, axis=1)[:, k - 1]
        for i in rows:
            cand = np.nonzero(D[i] >= thr[i])[0]
            order = cand[np.lexsort((cand, -D[i, cand]))][:k]
            out_i[c0 + i] = order
            out_d[c0 + i] = D[i, order]
    return out_i, out_d


class _Node:
    __slots__ = ("lo", "hi", "pts", "kids", "lam", "parent")


def _kdtree(P: np.ndarray, leaf_size: int) -> _Node:
    """kd-tree: split on the widest box dimension (lower index on ties), left
    child = the floor(n/2) smallest points on it (ties by index)."""
    def make(idx, parent):
        nd = _Node()
        X = P[idx]
        nd.lo, nd.hi = X.min(axis=0), X.max(axis=0)
        c = 0.5 * (nd.lo + nd.hi)
        nd.lam = float(np.sqrt(((X - c) ** 2).sum(axis=1)).max())
        nd.parent = parent
        nd.pts = idx
        nd.kids = []
        if len(idx) > leaf_size:
            dim = int(np.argmax(nd.hi - nd.lo))
            order = idx[np.lexsort((idx, P[idx, dim]))]
            h = len(idx) // 2
            nd.kids = [make(order[:h], nd), make(order[h:], nd)]
        return nd
    return make(np.arange(P.shape[0], dtype=np.int64), None)


def _dmax(a: _Node, b: _Node) -> float:
    """Largest distance between the two boxes."""
    g = np.maximum(np.abs(a.lo - b.hi), np.abs(a.hi - b.lo))
    return float(np.sqrt((g * g).sum()))


def kfn_dualtree(ref: np.ndarray, query: Optional[np.ndarray], k: int, leaf_size: int = 4,
                 strict: bool = True, stats: Optional[dict] = None
                 ) -> Tuple[np.ndarray, np.ndarray]:
    """k-furthest neighbours by the dual-tree meta-algorithm with the inverted
    Score and BaseCase (small inputs only).  ``strict=False`` prunes at
    d_max == B' as well (kept to show that this loses ties)."""
    R = np.asarray(ref, dtype=np.float32).astype(np.float64)
    mono = query is None
    Q = R if mono else np.asarray(query, dtype=np.float32).astype(np.float64)
    n = Q.shape[0]
    tr, tq = _kdtree(R, leaf_size), _kdtree(Q, leaf_size)
    # each query's list: (d2, idx) pairs, best first
    lists = [[] for _ in range(n)]
    st = {"scores": 0, "prunes": 0, "basecases": 0}

    def kth(p: int) -> float:
        """D_p[k] as a distance: 0 while p has fewer than k candidates."""
        return float(np.sqrt(lists[p][k - 1][0])) if len(lists[p]) >= k else 0.0

    def bound(nq: _Node) -> float:
        b = 0.0
        a = nq
        while a is not None:
            ds = [kth(int(p)) for p in a.pts]
            b = max(b, min(ds), max(ds) - 2.0 * a.lam)
            a = a.parent
        return b

    def base_case(pq: int, pr: int):
        if mono and pq == pr:
            return
        st["basecases"] += 1
        t = Q[pq] - R[pr]
        d2 = 0.0
        for v in t:
            d2 = d2 + v * v
        L = lists[pq]
        key = (-d2, pr)
        if len(L) == k and not key < (-L[-1][0], L[-1][1]):
            return
        L.append((d2, pr))
        L.sort(key=lambda e: (-e[0], e[1]))
        del L[k:]

    def traverse(nq: _Node, nr: _Node):
        st["scores"] += 1
        dm, b = _dmax(nq, nr), bound(nq)
        if dm < b or (not strict and dm <= b and b > 0.0):
            st["prunes"] += 1
            return
        if not nq.kids and not nr.kids:
            for pq in nq.pts:
                for pr in nr.pts:
                    base_case(int(pq), int(pr))
            return
        # split the node that has children (the query node when both do)
        if nq.kids:
            kids = [(c, nr) for c in nq.kids]
        else:
            kids = [(nq, c) for c in nr.kids]
        # farther pair first (the inverse of the kNN closer-first order)
        kids.sort(key=lambda ab: -_dmax(ab[0], ab[1]))
        for a, c in kids:
            traverse(a, c)

    traverse(tq, tr)
    if stats is not None:
        stats.update(st)
    # (a list can only come out short of k entries under strict=False)
    idx = np.array([[e[1] for e in L] + [-1] * (k - len(L)) for L in lists], dtype=np.int64)
    d2 = np.array([[e[0] for e in L] + [-1.0] * (k - len(L)) for L in lists], dtype=np.float64)
    return idx, d2
