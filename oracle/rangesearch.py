"""Float64 reference of range search -- TEST INFRASTRUCTURE ONLY.

Only the tests and ``bench.py``'s CPU legs (its ``cpu_baseline`` and
reference arm) import this module; the CUDA library never calls it.

Problem (Section 6, "Range Search"): given a range [delta1, delta2], for every
query p_q all reference points p_r with delta1 <= ||p_q - p_r|| <= delta2
(both ends inclusive); the lists are not ordered.  Readings:

* the distance is sqrt of the float64 sum of (q_j - r_j)^2 over j, left to
  right from the float32 inputs, with the correctly rounded square root, and
  it is compared with delta1 and delta2 as float64 values;
* a monochromatic query never returns itself (by index);
* the oracle lists each query's neighbours by ascending index (its own
  canonical order; the problem's lists are sets).

``range_brute`` is that definition written out.  ``range_dualtree`` is the
meta-algorithm of Section 2 (Algorithm 1's depth-first traversal) with the
range-search BaseCase and Score, on kd-trees (pure Python, small inputs), kept
as an independent check of the definition.  Its Score prunes a node pair when
no pair of points in it can lie in the range: d_min > delta2 or
d_max < delta1.  The printed Score keeps a pair only when
delta1 <= d_min <= delta2, which also prunes pairs with d_min < delta1 <=
d_max whose points can still lie in the range; ``literal=True`` uses it, to
show what it loses.
"""
from __future__ import annotations

from typing import Optional, Tuple

import numpy as np

from .kfn import _d2_rows, _kdtree


def range_brute(ref: np.ndarray, query: Optional[np.ndarray], d_lo: float, d_hi: float,
                chunk: int = 256) -> Tuple[np.ndarray, np.ndarray, np.ndarray]:
    """All pairs within [d_lo, d_hi].  Returns (offsets int64 (n + 1),
    idx int64 (total), dist float64 (total)); query i's neighbours are
    idx[offsets[i]:offsets[i + 1]], by ascending index."""
    R = np.asarray(ref, dtype=np.float32).astype(np.float64)
    mono = query is None
    Q = R if mono else np.asarray(query, dtype=np.float32).astype(np.float64)
    n = Q.shape[0]
    counts = np.zeros(n + 1, dtype=np.int64)
    parts_i, parts_d = [], []
    for c0 in range(0, n, chunk):
        D = np.sqrt(_d2_rows(Q[c0:c0 + chunk], R))
        inside = (D >= d_lo) & (D <= d_hi)
        if mono:
            rows = np.arange(D.shape[0])
            inside[rows, c0 + rows] = False
        for i in range(D.shape[0]):
            j = np.nonzero(inside[i])[0]
            counts[c0 + i + 1] = len(j)
            parts_i.append(j)
            parts_d.append(D[i, j])
    offsets = np.cumsum(counts)
    idx = np.concatenate(parts_i) if parts_i else np.zeros(0, dtype=np.int64)
    dist = np.concatenate(parts_d) if parts_d else np.zeros(0)
    return offsets, idx.astype(np.int64), dist


def _dmin_dmax(a, b) -> Tuple[float, float]:
    gmin = np.maximum(np.maximum(a.lo - b.hi, b.lo - a.hi), 0.0)
    gmax = np.maximum(np.abs(a.lo - b.hi), np.abs(a.hi - b.lo))
    return float(np.sqrt((gmin * gmin).sum())), float(np.sqrt((gmax * gmax).sum()))


def range_dualtree(ref: np.ndarray, query: Optional[np.ndarray], d_lo: float, d_hi: float,
                   leaf_size: int = 4, literal: bool = False, stats: Optional[dict] = None
                   ) -> Tuple[np.ndarray, np.ndarray, np.ndarray]:
    """Range search by the dual-tree meta-algorithm (small inputs only); the
    same output as range_brute."""
    R = np.asarray(ref, dtype=np.float32).astype(np.float64)
    mono = query is None
    Q = R if mono else np.asarray(query, dtype=np.float32).astype(np.float64)
    n = Q.shape[0]
    tr, tq = _kdtree(R, leaf_size), _kdtree(Q, leaf_size)
    found = [dict() for _ in range(n)]
    st = {"scores": 0, "prunes": 0, "basecases": 0}

    def base_case(pq: int, pr: int):
        if mono and pq == pr:
            return
        st["basecases"] += 1
        t = Q[pq] - R[pr]
        d2 = 0.0
        for v in t:
            d2 = d2 + v * v
        d = float(np.sqrt(d2))
        if d_lo <= d <= d_hi:
            found[pq][pr] = d

    def traverse(nq, nr):
        st["scores"] += 1
        dmin, dmax = _dmin_dmax(nq, nr)
        pruned = not (d_lo <= dmin <= d_hi) if literal else (dmin > d_hi or dmax < d_lo)
        if pruned:
            st["prunes"] += 1
            return
        if not nq.kids and not nr.kids:
            for pq in nq.pts:
                for pr in nr.pts:
                    base_case(int(pq), int(pr))
            return
        kids = [(c, nr) for c in nq.kids] if nq.kids else [(nq, c) for c in nr.kids]
        for a, c in kids:
            traverse(a, c)

    traverse(tq, tr)
    if stats is not None:
        stats.update(st)
    counts = np.zeros(n + 1, dtype=np.int64)
    idx, dist = [], []
    for i in range(n):
        js = sorted(found[i])
        counts[i + 1] = len(js)
        idx.extend(js)
        dist.extend(found[i][j] for j in js)
    return np.cumsum(counts), np.array(idx, dtype=np.int64), np.array(dist, dtype=np.float64)
