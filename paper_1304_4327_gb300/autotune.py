"""Autotuner for the kNN search: per problem class, the leaf size of the
trees and the number of queries per block (the M side of a BaseCase tile).

A class is (width bucket, log2 of the reference size, log2 of the query
size, k, precision).  The first time a class is seen, each candidate
(leaf size x queries per block) builds the problem's trees and runs the
search, timed with CUDA events (best of `repeats`). The fastest candidate is
kept, in memory and, when a path is given, in a JSON file that later runs
load.  The work itself runs in the library; this module only chooses its
parameters.
"""
from __future__ import annotations

import json
import math
import os
from typing import Dict, Iterable, List, Optional, Sequence, Tuple

LEAVES = (8, 16, 32, 64)
BLOCKS = (32, 64, 128, 256, 512)


def width_bucket(d: int) -> int:
    for b in (4, 8, 16, 32, 64):
        if d <= b:
            return b
    raise ValueError("d must be at most 64")


def problem_class(n_ref: int, n_query: int, d: int, k: int, precision: str) -> str:
    """The cache key of a problem: sizes enter by their power of two."""
    lr = int(math.floor(math.log2(max(n_ref, 1))))
    lq = int(math.floor(math.log2(max(n_query, 1))))
    return f"d{width_bucket(d)}/r{lr}/q{lq}/k{k}/{precision}"


class Autotuner:
    def __init__(self, path: Optional[str] = None, leaves: Sequence[int] = LEAVES,
                 blocks: Sequence[int] = BLOCKS, repeats: int = 2):
        self.path = path
        self.leaves = tuple(leaves)
        self.blocks = tuple(blocks)
        self.repeats = repeats
        self.table: Dict[str, Tuple[int, int]] = {}
        self.timings: Dict[str, Dict[str, float]] = {}
        if path and os.path.exists(path):
            with open(path) as f:
                raw = json.load(f)
            self.table = {k: (int(v[0]), int(v[1])) for k, v in raw.items()}

    def save(self) -> None:
        if not self.path:
            return
        tmp = self.path + ".tmp"
        with open(tmp, "w") as f:
            json.dump({k: list(v) for k, v in sorted(self.table.items())}, f, indent=1)
        os.replace(tmp, self.path)

    def _measure(self, dt, ref, query, k: int, precision: str) -> Dict[Tuple[int, int], float]:
        import torch
        stream = torch.cuda.current_stream()
        out: Dict[Tuple[int, int], float] = {}
        for leaf in self.leaves:
            for qb in self.blocks:
                best = float("inf")
                for _ in range(self.repeats):
                    e0 = torch.cuda.Event(enable_timing=True)
                    e1 = torch.cuda.Event(enable_timing=True)
                    e0.record(stream)
                    tr = dt.dtree_build(ref, leaf)
                    tq = None if query is None else dt.dtree_build(query, leaf)
                    try:
                        dt.dtree_knn(tq, tr, k, precision=precision, query_block=qb)
                    finally:
                        tr.free()
                        if tq is not None:
                            tq.free()
                    e1.record(stream)
                    e1.synchronize()
                    best = min(best, e0.elapsed_time(e1))
                out[(leaf, qb)] = best
        return out

    def choose(self, ref, query, k: int, precision: str = "fp32") -> Tuple[int, int]:
        """(leaf size, queries per block) for this problem's class; measured on
        this problem the first time the class is seen."""
        n_ref, d = int(ref.shape[0]), int(ref.shape[1])
        n_query = n_ref if query is None else int(query.shape[0])
        key = problem_class(n_ref, n_query, d, k, precision)
        if key not in self.table:
            from . import dtree as dt
            times = self._measure(dt, ref, query, k, precision)
            self.table[key] = min(times, key=times.get)
            self.timings[key] = {f"{a}/{b}": t for (a, b), t in times.items()}
            self.save()
        return self.table[key]

    def choose_batch(self, problems: Iterable[Tuple[object, Optional[object], int]],
                     precision: str = "fp32") -> List[Tuple[int, int]]:
        return [self.choose(ref, query, k, precision) for ref, query, k in problems]


def run_batch(problems: Sequence[Tuple[object, Optional[object], int]], precision: str = "fp32",
              tuner: Optional[Autotuner] = None, **knn_opts):
    """Build every problem's trees with its tuned leaf size and answer all of
    them in one dtree_knn_batch call with their tuned block sizes.
    ``problems``: (ref points, query points or None, k) device tensors;
    ``knn_opts`` go to dtree_knn_batch (seed_points, cap_leaves, ...).
    Returns one (idx, dist) pair per problem."""
    from . import dtree as dt
    tuner = tuner or Autotuner()
    choice = tuner.choose_batch(problems, precision)
    trees = []
    try:
        for (ref, query, k), (leaf, qb) in zip(problems, choice):
            tr = dt.dtree_build(ref, leaf)
            tq = None if query is None else dt.dtree_build(query, leaf)
            trees.append((tq, tr, k, qb))
        return dt.dtree_knn_batch(trees, precision=precision, **knn_opts)
    finally:
        for tq, tr, _, _ in trees:
            tr.free()
            if tq is not None:
                tq.free()
