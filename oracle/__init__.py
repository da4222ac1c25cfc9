"""CPU oracle for exact k-nearest-neighbour search -- TEST INFRASTRUCTURE ONLY.

Only the tests, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` import this package.  The CUDA library never links, loads or calls
it, and it imports nothing from the CUDA package (the seeded input generators
live in their own module and hold none of the method's arithmetic).

The C source (``dtree_oracle.c``) is plain IEEE double precision compiled with
``-ffp-contract=off``; see its header for the paper passages and the readings
of the paper it follows.  ``mlp.py`` holds the double-precision reference of
the learned proposal's network, ``kfn.py`` the k-furthest-neighbour problem
(its brute-force definition and the inverted dual-tree), and
``rangesearch.py`` range search (its definition and the dual-tree with the
range Score), and ``emst.py`` the Euclidean minimum spanning tree (Kruskal
and Prim under one total edge order).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from typing import Optional, Tuple

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "dtree_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")

BOUND_SOUND, BOUND_LITERAL, BOUND_B1, BOUND_NONE = 0, 1, 2, 3
DMIN_KINDS = {"box": 0, "ball": 1, "both": 2}
STAT_NAMES = ("scores", "prunes", "leaf_pairs", "basecases", "audit_prune",
              "audit_bound", "order", "qnodes", "incomplete")

_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle with gcc into oracle/liboracle.so (host architecture)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        cmd = ["gcc", "-O2", "-fopenmp", "-ffp-contract=off", "-fPIC", "-shared",
               "-o", _LIB + ".tmp", _SRC, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(_LIB + ".tmp", _LIB)
    return _LIB


def _load():
    global _lib
    if _lib is None:
        build()
        lib = ctypes.CDLL(_LIB)
        P, I64, I32 = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int32
        lib.oracle_knn_brute.argtypes = [P, I64, P, I64, I32, I32, P, P, P]
        lib.oracle_knn_dualtree.argtypes = [P, I64, P, I64, I32, I32, I32, I32, I32, I32, I32,
                                            P, P, P, P, P]
        lib.oracle_allnn_gray.argtypes = [P, I64, P, I64, I32, I32, I32, I32, P, P]
        lib.oracle_kdtree_check.argtypes = [P, I64, I32, I32, P]
        lib.oracle_set_threads.argtypes = [I32]
        for f in (lib.oracle_knn_brute, lib.oracle_knn_dualtree, lib.oracle_allnn_gray,
                  lib.oracle_kdtree_check, lib.oracle_set_threads):
            f.restype = ctypes.c_int
        _lib = lib
    return _lib


def _f32(a: np.ndarray) -> np.ndarray:
    a = np.ascontiguousarray(a, dtype=np.float32)
    if a.ndim != 2:
        raise ValueError("points must be a 2-D (n, d) array")
    return a


def _ptr(a: Optional[np.ndarray]):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


def set_threads(n: int) -> int:
    """Set the OpenMP thread count (n <= 0 keeps the default); returns the count in use."""
    return int(_load().oracle_set_threads(int(n)))


def knn_brute(ref: np.ndarray, query: Optional[np.ndarray], k: int,
              self_idx: Optional[np.ndarray] = None) -> Tuple[np.ndarray, np.ndarray]:
    """Exact kNN by comparing every pair (the definition of the result).

    ``query is None`` means monochromatic: the queries are the references and
    query i never returns reference i.  ``self_idx`` (int64, one per query)
    names the reference each query must skip (-1 for none), for sampled
    monochromatic queries.  Returns (idx int64 (n, k), d2 float64 (n, k))
    ascending by (squared distance, index).
    """
    lib = _load()
    r = _f32(ref)
    if query is None:
        q = r
        self_idx = np.arange(r.shape[0], dtype=np.int64)
    else:
        q = _f32(query)
    if q.shape[1] != r.shape[1]:
        raise ValueError("dimension mismatch")
    if self_idx is not None:
        self_idx = np.ascontiguousarray(self_idx, dtype=np.int64)
    n = q.shape[0]
    idx = np.empty((n, k), dtype=np.int64)
    d2 = np.empty((n, k), dtype=np.float64)
    rc = lib.oracle_knn_brute(_ptr(q), n, _ptr(r), r.shape[0], r.shape[1], k,
                              _ptr(self_idx), _ptr(idx), _ptr(d2))
    if rc != 0:
        raise ValueError(f"oracle_knn_brute failed ({rc})")
    return idx, d2


def knn_dualtree(ref: np.ndarray, query: Optional[np.ndarray], k: int, leaf_size: int = 20,
                 bound: int = BOUND_SOUND, par_depth: int = 0,
                 truth: Optional[Tuple[np.ndarray, np.ndarray]] = None, dmin: str = "box"):
    """Serial kd-tree dual-tree kNN (Algorithms 1, 2, 3 with the bound B).

    ``dmin`` is Score's node lower bound: "box" (the kd-tree), "ball" (balls
    of radius lambda around the box centres: a ball tree over the same
    splits) or "both" (the larger).

    Returns (idx, d2, stats dict).  With ``truth`` = brute-force (idx, d2) the
    audit counters ``audit_prune`` (pruned pairs that held a true neighbour)
    and ``audit_bound`` (Score calls with B(N_q) below a true k-th distance
    in the node) are filled.
    """
    lib = _load()
    r = _f32(ref)
    mono = query is None
    q = r if mono else _f32(query)
    n = q.shape[0]
    idx = np.empty((n, k), dtype=np.int64)
    d2 = np.empty((n, k), dtype=np.float64)
    st = np.zeros(len(STAT_NAMES), dtype=np.int64)
    ti = td = None
    if truth is not None:
        ti = np.ascontiguousarray(truth[0], dtype=np.int64)
        td = np.ascontiguousarray(truth[1], dtype=np.float64)
    rc = lib.oracle_knn_dualtree(None if mono else _ptr(q), n, _ptr(r), r.shape[0], r.shape[1],
                                 k, int(mono), leaf_size, bound, DMIN_KINDS[dmin], par_depth,
                                 _ptr(ti), _ptr(td),
                                 _ptr(idx), _ptr(d2), _ptr(st))
    if rc != 0:
        raise ValueError(f"oracle_knn_dualtree failed ({rc})")
    return idx, d2, dict(zip(STAT_NAMES, (int(v) for v in st)))


def allnn_gray(ref: np.ndarray, query: Optional[np.ndarray], leaf_size: int = 20,
               variant: int = 0) -> Tuple[np.ndarray, np.ndarray]:
    """Gray's all-nearest-neighbours (Algorithm 4, k = 1)."""
    lib = _load()
    r = _f32(ref)
    mono = query is None
    q = r if mono else _f32(query)
    n = q.shape[0]
    idx = np.empty(n, dtype=np.int64)
    d2 = np.empty(n, dtype=np.float64)
    rc = lib.oracle_allnn_gray(None if mono else _ptr(q), n, _ptr(r), r.shape[0], r.shape[1],
                               int(mono), leaf_size, variant, _ptr(idx), _ptr(d2))
    if rc != 0:
        raise ValueError(f"oracle_allnn_gray failed ({rc})")
    return idx, d2


def kdtree_check(pts: np.ndarray, leaf_size: int):
    """(nodes, leaves, max depth, violations) of the oracle's kd-tree."""
    p = _f32(pts)
    out = np.zeros(4, dtype=np.int64)
    rc = _load().oracle_kdtree_check(_ptr(p), p.shape[0], p.shape[1], leaf_size, _ptr(out))
    if rc != 0:
        raise ValueError(f"oracle_kdtree_check failed ({rc})")
    return tuple(int(v) for v in out)
