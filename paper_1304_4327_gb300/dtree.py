"""Python binding of the C ABI declared in include/dtree.h.

Argument marshalling only: every step of the search runs in the CUDA library
(``libdtree.so``).  PyTorch supplies device memory and the current stream.
Importing this module loads the library and fails loudly if it is missing;
there is no CPU fallback.
"""
from __future__ import annotations

import ctypes
import os
from typing import Optional, Tuple

import torch

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libdtree.so")

DTREE_OK = 0
PRECISIONS = {"fp32": 0, "tf32": 1, "bf16": 2}
BOUNDS = {"box": 0, "ball": 1, "both": 2}
_I32, _I64, _P = ctypes.c_int32, ctypes.c_int64, ctypes.c_void_p


class dtree_opts(ctypes.Structure):
    _fields_ = [("leaf_size", _I32), ("precision", _I32), ("query_block", _I32),
                ("seed_points", _I32), ("proposal", _I32), ("spin_budget", _I32),
                ("cap_leaves", _I32), ("bound", _I32), ("reserved", _I32 * 8)]


STAT_FIELDS = ("node_pairs_scored", "node_pairs_pruned", "leaf_pairs_emitted",
               "leaf_pairs_skipped", "leaf_pairs_evaluated", "point_pairs",
               "rerank_candidates", "fallback_queries", "query_blocks", "kernel_launches",
               "ns_seed", "ns_traverse", "ns_basecase", "ns_fallback", "fallback64_queries",
               "seed_point_pairs")


class dtree_stats(ctypes.Structure):
    _fields_ = [(f, _I64) for f in STAT_FIELDS]


class dtree_problem(ctypes.Structure):
    _fields_ = [("query", _P), ("ref", _P), ("k", _I32), ("query_block", _I32),
                ("out_idx", _P), ("out_dist", _P)]


class dtree_train_opts(ctypes.Structure):
    _fields_ = [("epochs", _I32), ("batch", _I32), ("lr", ctypes.c_float),
                ("example_queries", _I32), ("seed_points", _I32), ("seed", ctypes.c_uint32),
                ("loss_out", ctypes.POINTER(ctypes.c_float)), ("loss_out_len", _I32),
                ("precision", _I32), ("reserved", _I32 * 7)]


class DTreeError(RuntimeError):
    def __init__(self, status: int, where: str):
        self.status = status
        super().__init__(f"{where}: {error_string(status)} ({status})")


def _load() -> ctypes.CDLL:
    if not os.path.exists(LIB_PATH):
        raise ImportError(
            f"{LIB_PATH} is missing: build it with paper_1304_4327_gb300.build.build() "
            "(there is no CPU fallback)")
    lib = ctypes.CDLL(LIB_PATH)
    lib.dtree_build.argtypes = [_P, _I64, _I32, ctypes.POINTER(dtree_opts), _P, ctypes.POINTER(_P)]
    lib.dtree_knn.argtypes = [_P, _P, _I32, _P, _P, ctypes.POINTER(dtree_opts), _P,
                              ctypes.POINTER(dtree_stats)]
    lib.dtree_free.argtypes = [_P]
    lib.dtree_free.restype = None
    lib.dtree_size.argtypes = [_P]
    lib.dtree_size.restype = _I64
    lib.dtree_dim.argtypes = [_P]
    lib.dtree_dim.restype = _I32
    lib.dtree_depth.argtypes = [_P]
    lib.dtree_depth.restype = _I32
    lib.dtree_leaf_count.argtypes = [_P]
    lib.dtree_leaf_count.restype = _I64
    lib.dtree_export.argtypes = [_P, _P, _P, _P, _P, _P, _P]
    lib.dtree_error_string.argtypes = [ctypes.c_int]
    lib.dtree_error_string.restype = ctypes.c_char_p
    lib.dtree_debug_mma.argtypes = [_P, _P, _I32, _I32, _P, _P]
    lib.dtree_debug_mma.restype = ctypes.c_int
    lib.dtree_debug_tmem_min.argtypes = [_P, _P, _I32, _I32, _P, _P, _P, _P]
    lib.dtree_debug_tmem_min.restype = ctypes.c_int
    lib.dtree_debug_tc_timers.argtypes = [_P]
    lib.dtree_debug_tc_timers.restype = ctypes.c_int
    lib.dtree_debug_tc_stall.argtypes = [_I32]
    lib.dtree_debug_tc_stall.restype = ctypes.c_int
    lib.dtree_launch_count.argtypes = []
    lib.dtree_launch_count.restype = _I64
    lib.dtree_alloc_count.argtypes = []
    lib.dtree_alloc_count.restype = _I64
    lib.dtree_knn_noalloc.argtypes = [_P, _P, _I32, _P, _P, ctypes.POINTER(dtree_opts), _P]
    lib.dtree_kfn.argtypes = [_P, _P, _I32, _P, _P, ctypes.POINTER(dtree_opts), _P,
                              ctypes.POINTER(dtree_stats)]
    lib.dtree_range_count.argtypes = [_P, _P, ctypes.c_double, ctypes.c_double, _P,
                                      ctypes.POINTER(_I64), ctypes.POINTER(dtree_opts), _P,
                                      ctypes.POINTER(dtree_stats)]
    lib.dtree_range_fill.argtypes = [_P, _P, ctypes.c_double, ctypes.c_double, _P, _P, _P,
                                     ctypes.POINTER(dtree_opts), _P]
    lib.dtree_emst.argtypes = [_P, _P, _P, ctypes.POINTER(dtree_opts), _P, ctypes.POINTER(dtree_stats)]
    lib.dtree_knn_batch.argtypes = [_I32, ctypes.POINTER(dtree_problem), ctypes.POINTER(dtree_opts),
                                    _P, ctypes.POINTER(dtree_stats)]
    lib.dtree_proposal_train.argtypes = [_P, _P, _I32, ctypes.POINTER(dtree_train_opts), _P,
                                         ctypes.POINTER(_P)]
    lib.dtree_proposal_train.restype = ctypes.c_int
    lib.dtree_model_free.argtypes = [_P]
    lib.dtree_model_free.restype = None
    lib.dtree_model_classes.argtypes = [_P]
    lib.dtree_model_classes.restype = ctypes.c_int
    lib.dtree_model_save.argtypes = [_P, ctypes.c_char_p, _P]
    lib.dtree_model_save.restype = ctypes.c_int
    lib.dtree_model_load.argtypes = [ctypes.c_char_p, _P, _P, ctypes.POINTER(_P)]
    lib.dtree_model_load.restype = ctypes.c_int
    lib.dtree_attach_proposal.argtypes = [_P, _P]
    lib.dtree_attach_proposal.restype = ctypes.c_int
    lib.dtree_mlp_loss_grad.argtypes = [_I32, _I32, ctypes.POINTER(_P), _P, _P, _I32,
                                        ctypes.POINTER(ctypes.c_float), ctypes.POINTER(_P), _P]
    lib.dtree_mlp_loss_grad.restype = ctypes.c_int
    for f in (lib.dtree_build, lib.dtree_knn, lib.dtree_export, lib.dtree_knn_noalloc,
              lib.dtree_knn_batch):
        f.restype = ctypes.c_int
    return lib


_lib = _load()


def error_string(status: int) -> str:
    return _lib.dtree_error_string(int(status)).decode()


def launch_count() -> int:
    """Kernels launched by the library in this process so far."""
    return int(_lib.dtree_launch_count())


def alloc_count() -> int:
    """Device allocations the library has made in this process so far."""
    return int(_lib.dtree_alloc_count())


def _stream(stream) -> ctypes.c_void_p:
    if stream is None:
        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(stream.cuda_stream)


def _opts(**kw) -> dtree_opts:
    o = dtree_opts()
    for key, val in kw.items():
        if val is not None:
            setattr(o, key, int(val))
    return o


def _check_points(x: torch.Tensor, name: str) -> torch.Tensor:
    if not isinstance(x, torch.Tensor) or not x.is_cuda:
        raise TypeError(f"{name} must be a CUDA tensor")
    if x.dtype != torch.float32 or x.dim() != 2:
        raise TypeError(f"{name} must be a 2-D float32 tensor")
    return x.contiguous()


class Tree:
    """Owning wrapper of a dtree_t* handle."""

    def __init__(self, handle: int):
        self.handle = ctypes.c_void_p(handle)

    @property
    def n(self) -> int:
        return int(_lib.dtree_size(self.handle))

    @property
    def d(self) -> int:
        return int(_lib.dtree_dim(self.handle))

    @property
    def depth(self) -> int:
        return int(_lib.dtree_depth(self.handle))

    @property
    def leaves(self) -> int:
        return int(_lib.dtree_leaf_count(self.handle))

    def free(self) -> None:
        if self.handle and self.handle.value:
            _lib.dtree_free(self.handle)
            self.handle = ctypes.c_void_p(None)

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass


def dtree_build(points: torch.Tensor, leaf_size: int = 32, stream=None) -> Tree:
    """Build a kd-tree on the device (see dtree_build in include/dtree.h)."""
    pts = _check_points(points, "points")
    out = ctypes.c_void_p()
    o = _opts(leaf_size=leaf_size)
    rc = _lib.dtree_build(ctypes.c_void_p(pts.data_ptr()), pts.shape[0], pts.shape[1],
                          ctypes.byref(o), _stream(stream), ctypes.byref(out))
    if rc != DTREE_OK:
        raise DTreeError(rc, "dtree_build")
    return Tree(out.value)


def dtree_knn(query: Optional[Tree], ref: Tree, k: int, precision: str = "fp32",
              query_block: int = 0, seed_points: int = 0, out_idx: Optional[torch.Tensor] = None,
              out_dist: Optional[torch.Tensor] = None, stream=None, with_stats: bool = False,
              proposal: int = 0, cap_leaves: int = 0, spin_budget: int = 0, bound: str = "box"):
    """Exact kNN of every point of ``query`` (None = monochromatic) in ``ref``.

    Returns (idx int64 (n_q, k), dist float32 (n_q, k)) on the device, plus a
    dict of counters when ``with_stats``.  ``cap_leaves``: leaves of each
    query's cap search (0: the library's default, -1: no cap pass).
    ``bound``: the node lower bound d_min, "box", "ball" or "both" (see dtree.h).
    """
    nq = ref.n if query is None else query.n
    dev = torch.device("cuda", torch.cuda.current_device())
    if k <= 0:  # let the library report the invalid k
        rc = _lib.dtree_knn(None if query is None else query.handle, ref.handle, int(k), None,
                            None, None, _stream(stream), None)
        raise DTreeError(rc, "dtree_knn")
    if out_idx is None:
        out_idx = torch.empty((nq, k), dtype=torch.int64, device=dev)
    if out_dist is None:
        out_dist = torch.empty((nq, k), dtype=torch.float32, device=dev)
    if out_idx.shape != (nq, k) or out_idx.dtype != torch.int64 or not out_idx.is_contiguous():
        raise ValueError("out_idx must be a contiguous int64 (n_q, k) tensor")
    if out_dist.shape != (nq, k) or out_dist.dtype != torch.float32 or not out_dist.is_contiguous():
        raise ValueError("out_dist must be a contiguous float32 (n_q, k) tensor")
    o = _opts(precision=PRECISIONS[precision], query_block=query_block, seed_points=seed_points,
              proposal=proposal, cap_leaves=cap_leaves, spin_budget=spin_budget, bound=BOUNDS[bound])
    st = dtree_stats()
    rc = _lib.dtree_knn(None if query is None else query.handle, ref.handle, int(k),
                        ctypes.c_void_p(out_idx.data_ptr()), ctypes.c_void_p(out_dist.data_ptr()),
                        ctypes.byref(o), _stream(stream), ctypes.byref(st) if with_stats else None)
    if rc != DTREE_OK:
        raise DTreeError(rc, "dtree_knn")
    if with_stats:
        return out_idx, out_dist, {f: int(getattr(st, f)) for f in STAT_FIELDS}
    return out_idx, out_dist


def dtree_knn_batch(problems, precision: str = "fp32", query_block: int = 0,
                    seed_points: int = 0, stream=None, with_stats: bool = False,
                    proposal: int = 0, cap_leaves: int = 0, spin_budget: int = 0):
    """Many independent kNN problems in one call.

    ``problems``: a sequence of (query Tree or None, ref Tree, k) or
    (query, ref, k, query_block).  Returns a list of (idx, dist) device
    tensors, one pair per problem (plus a dict of counters summed over the
    batch when ``with_stats``).
    """
    dev = torch.device("cuda", torch.cuda.current_device())
    n = len(problems)
    arr = (dtree_problem * max(n, 1))()
    outs = []
    for i, pr in enumerate(problems):
        query, ref, k = pr[0], pr[1], int(pr[2])
        qb = int(pr[3]) if len(pr) > 3 else 0
        nq = ref.n if query is None else query.n
        kk = max(k, 0)
        oi = torch.empty((nq, kk), dtype=torch.int64, device=dev)
        od = torch.empty((nq, kk), dtype=torch.float32, device=dev)
        outs.append((oi, od))
        arr[i].query = None if query is None else query.handle
        arr[i].ref = ref.handle
        arr[i].k = k
        arr[i].query_block = qb
        arr[i].out_idx = oi.data_ptr() if oi.numel() else None
        arr[i].out_dist = od.data_ptr() if od.numel() else None
    o = _opts(precision=PRECISIONS[precision], query_block=query_block, seed_points=seed_points,
              proposal=proposal, cap_leaves=cap_leaves, spin_budget=spin_budget)
    st = dtree_stats()
    rc = _lib.dtree_knn_batch(n, arr, ctypes.byref(o), _stream(stream),
                              ctypes.byref(st) if with_stats else None)
    if rc != DTREE_OK:
        raise DTreeError(rc, "dtree_knn_batch")
    if with_stats:
        return outs, {f: int(getattr(st, f)) for f in STAT_FIELDS}
    return outs


class Model:
    """A trained leaf proposal (library-owned; freed by free() or on collection)."""

    def __init__(self, handle: int, losses):
        self.handle = handle
        self.losses = losses

    @property
    def classes(self) -> int:
        return int(_lib.dtree_model_classes(self.handle))

    def free(self) -> None:
        if self.handle:
            _lib.dtree_model_free(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass


def dtree_proposal_train(ref: Tree, train: Tree, k: int, epochs: int = 0, batch: int = 0,
                         lr: float = 0.0, example_queries: int = 0, seed_points: int = 0,
                         seed: int = 0, stream=None, precision: str = "fp32") -> Model:
    """Train a leaf proposal for ``ref`` on the method's own kNN answers for the
    points of ``train`` (see dtree.h; ``precision`` is that search's, the answers
    are exact at each); returns the model and its per-epoch losses."""
    n_ep = epochs if epochs > 0 else 20
    losses = (ctypes.c_float * n_ep)()
    o = dtree_train_opts(epochs=epochs, batch=batch, lr=lr, example_queries=example_queries,
                         seed_points=seed_points, seed=seed, loss_out=losses, loss_out_len=n_ep,
                         precision=PRECISIONS[precision])
    h = _P()
    rc = _lib.dtree_proposal_train(ref.handle, train.handle, int(k), ctypes.byref(o),
                                   _stream(stream), ctypes.byref(h))
    if rc != DTREE_OK:
        raise DTreeError(rc, "dtree_proposal_train")
    return Model(h.value, [float(x) for x in losses])


def dtree_model_save(model: Model, path: str, stream=None) -> None:
    """Write a trained proposal to ``path`` (see dtree.h for the format)."""
    rc = _lib.dtree_model_save(model.handle, os.fsencode(path), _stream(stream))
    if rc != DTREE_OK:
        raise DTreeError(rc, "dtree_model_save")


def dtree_model_load(path: str, ref: Optional[Tree], stream=None) -> Model:
    """Read a proposal saved by dtree_model_save for the reference tree ``ref``."""
    h = _P()
    rc = _lib.dtree_model_load(os.fsencode(path), None if ref is None else ref.handle,
                               None if ref is None else _stream(stream), ctypes.byref(h))
    if rc != DTREE_OK:
        raise DTreeError(rc, "dtree_model_load")
    return Model(h.value, [])


def dtree_attach_proposal(ref: Tree, model: Optional[Model]) -> None:
    rc = _lib.dtree_attach_proposal(ref.handle, None if model is None else model.handle)
    if rc != DTREE_OK:
        raise DTreeError(rc, "dtree_attach_proposal")
    ref._proposal = model  # keep the model alive while attached


def dtree_mlp_loss_grad(params, X: torch.Tensor, T: torch.Tensor, stream=None):
    """Loss and gradients of the proposal network (W1, b1, W2, b2, W3, b3 as
    float32 CUDA tensors) on inputs X (n x d) against targets T (n x C)."""
    params = [p.contiguous() for p in params]
    n, d = X.shape
    C = T.shape[1]
    grads = [torch.empty_like(p) for p in params]
    pp = (_P * 6)(*[p.data_ptr() for p in params])
    gp = (_P * 6)(*[g.data_ptr() for g in grads])
    loss = ctypes.c_float()
    rc = _lib.dtree_mlp_loss_grad(int(d), int(C), pp, X.contiguous().data_ptr(),
                                  T.contiguous().data_ptr(), int(n), ctypes.byref(loss), gp,
                                  _stream(stream))
    if rc != DTREE_OK:
        raise DTreeError(rc, "dtree_mlp_loss_grad")
    torch.cuda.current_stream().synchronize()
    return float(loss.value), grads


NOALLOC_MAX_QUERIES = 65536


def dtree_kfn(query: Optional[Tree], ref: Tree, k: int, out_idx: Optional[torch.Tensor] = None,
              out_dist: Optional[torch.Tensor] = None, stream=None, with_stats: bool = False,
              precision: str = "fp32"):
    """Exact k-furthest neighbours of every point of ``query`` (None =
    monochromatic) in ``ref``: (idx int64 (n_q, k), dist float32 (n_q, k)) on
    the device, descending by distance (ties by the lower index), plus a dict
    of counters when ``with_stats``."""
    nq = ref.n if query is None else query.n
    dev = torch.device("cuda", torch.cuda.current_device())
    kk = max(int(k), 0)
    if out_idx is None:
        out_idx = torch.empty((nq, kk), dtype=torch.int64, device=dev)
    if out_dist is None:
        out_dist = torch.empty((nq, kk), dtype=torch.float32, device=dev)
    if out_idx.shape != (nq, kk) or out_idx.dtype != torch.int64 or not out_idx.is_contiguous():
        raise ValueError("out_idx must be a contiguous int64 (n_q, k) tensor")
    if out_dist.shape != (nq, kk) or out_dist.dtype != torch.float32 or not out_dist.is_contiguous():
        raise ValueError("out_dist must be a contiguous float32 (n_q, k) tensor")
    o = _opts(precision=PRECISIONS[precision])
    st = dtree_stats()
    rc = _lib.dtree_kfn(None if query is None else query.handle, ref.handle, int(k),
                        ctypes.c_void_p(out_idx.data_ptr()) if out_idx.numel() else None,
                        ctypes.c_void_p(out_dist.data_ptr()) if out_dist.numel() else None,
                        ctypes.byref(o), _stream(stream), ctypes.byref(st) if with_stats else None)
    if rc != DTREE_OK:
        raise DTreeError(rc, "dtree_kfn")
    if with_stats:
        return out_idx, out_dist, {f: int(getattr(st, f)) for f in STAT_FIELDS}
    return out_idx, out_dist


def dtree_range(query: Optional[Tree], ref: Tree, d_lo: float, d_hi: float, stream=None,
                with_stats: bool = False, precision: str = "fp32"):
    """Exact range search: every reference point with d_lo <= distance <=
    d_hi for every point of ``query`` (None = monochromatic).  Returns
    (offsets int64 (n_q + 1), idx int64 (total), dist float32 (total)) on the
    device: query row i's neighbours are idx[offsets[i]:offsets[i + 1]] (a
    set, in the search's visit order), plus a dict of counters when
    ``with_stats``."""
    nq = ref.n if query is None else query.n
    dev = torch.device("cuda", torch.cuda.current_device())
    qh = None if query is None else query.handle
    offsets = torch.empty(nq + 1, dtype=torch.int64, device=dev)
    total = _I64(0)
    o = _opts(precision=PRECISIONS[precision])
    st = dtree_stats()
    rc = _lib.dtree_range_count(qh, ref.handle, float(d_lo), float(d_hi),
                                ctypes.c_void_p(offsets.data_ptr()), ctypes.byref(total),
                                ctypes.byref(o), _stream(stream),
                                ctypes.byref(st) if with_stats else None)
    if rc != DTREE_OK:
        raise DTreeError(rc, "dtree_range_count")
    n = int(total.value)
    idx = torch.empty(n, dtype=torch.int64, device=dev)
    dist = torch.empty(n, dtype=torch.float32, device=dev)
    if n > 0:
        rc = _lib.dtree_range_fill(qh, ref.handle, float(d_lo), float(d_hi),
                                   ctypes.c_void_p(offsets.data_ptr()), ctypes.c_void_p(idx.data_ptr()),
                                   ctypes.c_void_p(dist.data_ptr()), ctypes.byref(o), _stream(stream))
        if rc != DTREE_OK:
            raise DTreeError(rc, "dtree_range_fill")
    if with_stats:
        return offsets, idx, dist, {f: int(getattr(st, f)) for f in STAT_FIELDS}
    return offsets, idx, dist


def dtree_emst(tree: Tree, stream=None, with_stats: bool = False, precision: str = "fp32"):
    """The Euclidean minimum spanning tree of the tree's points (edges of equal
    length ordered by their endpoints' indices, so it is unique): (edges int64
    (n - 1, 2) as (lower, higher) caller row indices, dist float32 (n - 1)) on
    the device, in the order the rounds found them, plus a dict of counters
    when ``with_stats``."""
    n = tree.n
    dev = torch.device("cuda", torch.cuda.current_device())
    edges = torch.empty((max(n - 1, 0), 2), dtype=torch.int64, device=dev)
    dist = torch.empty(max(n - 1, 0), dtype=torch.float32, device=dev)
    o = _opts(precision=PRECISIONS[precision])
    st = dtree_stats()
    rc = _lib.dtree_emst(tree.handle, ctypes.c_void_p(edges.data_ptr()) if edges.numel() else None,
                         ctypes.c_void_p(dist.data_ptr()) if dist.numel() else None,
                         ctypes.byref(o), _stream(stream), ctypes.byref(st) if with_stats else None)
    if rc != DTREE_OK:
        raise DTreeError(rc, "dtree_emst")
    if with_stats:
        return edges, dist, {f: int(getattr(st, f)) for f in STAT_FIELDS}
    return edges, dist


def dtree_knn_noalloc(query: Optional[Tree], ref: Tree, k: int, out_idx: torch.Tensor,
                      out_dist: torch.Tensor, precision: str = "fp32", query_block: int = 0,
                      seed_points: int = 0, stream=None, cap_leaves: int = 0, bound: str = "box") -> None:
    """dtree_knn with no device allocation: the outputs are the caller's
    (contiguous int64 / float32 (n_q, k) tensors) and the library's scratch
    is a fixed static array.  Overlapping calls on one device race."""
    nq = ref.n if query is None else query.n
    if out_idx.shape != (nq, k) or out_idx.dtype != torch.int64 or not out_idx.is_contiguous():
        raise ValueError("out_idx must be a contiguous int64 (n_q, k) tensor")
    if out_dist.shape != (nq, k) or out_dist.dtype != torch.float32 or not out_dist.is_contiguous():
        raise ValueError("out_dist must be a contiguous float32 (n_q, k) tensor")
    o = _opts(precision=PRECISIONS[precision], query_block=query_block, seed_points=seed_points,
              cap_leaves=cap_leaves, bound=BOUNDS[bound])
    rc = _lib.dtree_knn_noalloc(None if query is None else query.handle, ref.handle, int(k),
                                ctypes.c_void_p(out_idx.data_ptr()),
                                ctypes.c_void_p(out_dist.data_ptr()), ctypes.byref(o),
                                _stream(stream))
    if rc != DTREE_OK:
        raise DTreeError(rc, "dtree_knn_noalloc")


def dtree_free(tree: Tree) -> None:
    tree.free()


def dtree_export(tree: Tree, stream=None) -> dict:
    """The tree's layout as device tensors (perm, box, lambda, begin, count)."""
    dev = torch.device("cuda", torch.cuda.current_device())
    nodes = 2 * tree.leaves - 1
    perm = torch.empty(tree.n, dtype=torch.int32, device=dev)
    box = torch.empty((nodes, 2, tree.d), dtype=torch.float32, device=dev)
    lam = torch.empty(nodes, dtype=torch.float32, device=dev)
    beg = torch.empty(nodes, dtype=torch.int32, device=dev)
    cnt = torch.empty(nodes, dtype=torch.int32, device=dev)
    rc = _lib.dtree_export(tree.handle, *(ctypes.c_void_p(t.data_ptr()) for t in (perm, box, lam, beg, cnt)),
                           _stream(stream))
    if rc != DTREE_OK:
        raise DTreeError(rc, "dtree_export")
    return {"perm": perm, "box": box, "lambda": lam, "begin": beg, "count": cnt}


def knn(ref_points: torch.Tensor, query_points: Optional[torch.Tensor], k: int,
        leaf_size: int = 32, **kw) -> Tuple[torch.Tensor, torch.Tensor]:
    """Build the tree(s), search, free: the one-call form of the API."""
    tr = dtree_build(ref_points, leaf_size)
    tq = None if query_points is None else dtree_build(query_points, leaf_size)
    try:
        return dtree_knn(tq, tr, k, **kw)
    finally:
        tr.free()
        if tq is not None:
            tq.free()


def dtree_debug_mma(A: torch.Tensor, B: torch.Tensor, fmt: str = "bf16", stream=None) -> torch.Tensor:
    """One 128 x 128 tensor-core tile, A (128, K) times B (128, K)^T (diagnostic)."""
    A = _check_points(A, "A")
    B = _check_points(B, "B")
    out = torch.empty((128, 128), dtype=torch.float32, device=A.device)
    rc = _lib.dtree_debug_mma(ctypes.c_void_p(A.data_ptr()), ctypes.c_void_p(B.data_ptr()),
                              A.shape[1], PRECISIONS[fmt], ctypes.c_void_p(out.data_ptr()),
                              _stream(stream))
    if rc != DTREE_OK:
        raise DTreeError(rc, "dtree_debug_mma")
    return out


TC_TIMERS = ("plan_window", "plan_wait", "plan_stage", "mma_wait", "epi_wait", "epi_work",
             "epi_rare_chunks", "epi_finish", "item_setup", "tiles", "items", "inserts", "epi_ld",
             "epi_loop", "epi_flush", "mma_wait_acc", "fail_sites", "epi_work_w2",
             "plan_copy", "copy_land")


def dtree_debug_tmem_min(A: torch.Tensor, B: torch.Tensor, fmt: str = "bf16", stream=None):
    """dtree_debug_mma's tile and the minima the tensor-core loads reduce to:
    (tile (128, 128), min over 32 columns (128, 4), min over 64 (128, 2))."""
    A = _check_points(A, "A")
    B = _check_points(B, "B")
    out = torch.empty((128, 128), dtype=torch.float32, device=A.device)
    m32 = torch.empty((128, 4), dtype=torch.float32, device=A.device)
    m64 = torch.empty((128, 2), dtype=torch.float32, device=A.device)
    rc = _lib.dtree_debug_tmem_min(ctypes.c_void_p(A.data_ptr()), ctypes.c_void_p(B.data_ptr()),
                                   A.shape[1], PRECISIONS[fmt], ctypes.c_void_p(out.data_ptr()),
                                   ctypes.c_void_p(m32.data_ptr()), ctypes.c_void_p(m64.data_ptr()),
                                   _stream(stream))
    if rc != DTREE_OK:
        raise DTreeError(rc, "dtree_debug_tmem_min")
    return out, m32, m64


def dtree_debug_tc_stall(on: bool) -> None:
    """Make every block of the tensor-core pass wait on a barrier that nothing
    completes (diagnostic of the bounded waits; see include/dtree.h)."""
    _lib.dtree_debug_tc_stall(1 if on else 0)


def dtree_debug_tc_timers(buf: Optional[torch.Tensor]) -> None:
    """Attach (or with None detach) a zeroed int64 CUDA tensor of 64 counters:
    0..31 for the main tensor-core pass, 32..63 for the seed pass."""
    if buf is not None and (buf.numel() < 64 or buf.dtype != torch.int64 or not buf.is_cuda):
        raise ValueError("the timer buffer must be a CUDA int64 tensor of at least 64 entries")
    _lib.dtree_debug_tc_timers(None if buf is None else ctypes.c_void_p(buf.data_ptr()))
