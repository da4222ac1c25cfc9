"""dtree_knn with Score's d_min as balls around the box centres (a ball tree
over the kd-tree's splits) or as the larger of boxes and balls: the lists
must equal the FP64 oracle's whatever the bound; only the pruning changes."""
import ctypes

import numpy as np
import pytest
import torch

from paper_1304_4327_gb300 import inputs
from parity import compare
from test_gpu_knn import run, truth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def dt():
    from paper_1304_4327_gb300 import build
    build.build()
    from paper_1304_4327_gb300 import dtree
    return dtree


@pytest.mark.parametrize("bound", ["ball", "both"])
@pytest.mark.parametrize("prec", ["fp32", "bf16"])
@pytest.mark.parametrize("d", [3, 16, 64])
@pytest.mark.parametrize("mono", [True, False])
def test_ball_bounds_match_the_oracle(dt, bound, prec, d, mono):
    R = inputs.gaussian(6001, d, 7100 + d)
    Q = None if mono else inputs.uniform(1503, d, 7200 + d) * 2 - 1
    for k in (1, 10):
        idx, dist = run(dt, R, Q, k, 16, precision=prec, bound=bound)
        ti, td = truth(R, Q, k)
        compare(idx, dist, ti, td, k)


@pytest.mark.parametrize("bound", ["box", "ball", "both"])
def test_bounds_on_the_mixture_agree_and_prune(dt, bound):
    W = inputs.gmm16(n_ref=200_000, n_query=20_000)
    idx, dist, st = run(dt, W.ref, W.query, W.k, W.leaf_size, stats=True, precision="bf16", bound=bound)
    ti, td = truth(W.ref, W.query, W.k)
    compare(idx, dist, ti, td, W.k)
    # well separated clusters: every bound prunes; boxes (alone or with the
    # balls) keep under half of the (block, leaf) pairs.  Balls alone are
    # much looser at d = 16: a kd leaf is a thin slab, and the ball around its
    # centre has the slab's half-diagonal as radius
    assert st["node_pairs_pruned"] > 0
    if bound != "ball":
        assert st["leaf_pairs_emitted"] < 0.5 * (20_000 / 100) * (200_000 / 32)


def test_ball_bound_at_d64_k50(dt):
    W = inputs.powerlaw64(n_ref=60_000, n_query=6_000)
    idx, dist = run(dt, W.ref, W.query, W.k, W.leaf_size, precision="bf16", bound="both")
    ti, td = truth(W.ref, W.query, W.k)
    r = compare(idx, dist, ti, td, W.k)
    assert r["exact"] + r["exempt"] == 6_000


def test_no_alloc_entry_takes_the_bound(dt):
    R = inputs.gaussian(30_000, 8, 7301)
    Q = inputs.gaussian(5_000, 8, 7302)
    tr = dt.dtree_build(torch.from_numpy(R).cuda(), 16)
    tq = dt.dtree_build(torch.from_numpy(Q).cuda(), 16)
    try:
        i0, d0 = dt.dtree_knn(tq, tr, 5, bound="ball")
        oi = torch.empty_like(i0)
        od = torch.empty_like(d0)
        dt.dtree_knn_noalloc(tq, tr, 5, oi, od, bound="ball")
        torch.cuda.synchronize()
        assert torch.equal(oi, i0) and torch.equal(od, d0)
    finally:
        tr.free()
        tq.free()


def test_an_unknown_bound_is_rejected(dt):
    R = torch.from_numpy(inputs.uniform(2000, 3, 7303)).cuda()
    tr = dt.dtree_build(R, 16)
    try:
        oi = torch.empty((2000, 3), dtype=torch.int64, device="cuda")
        od = torch.empty((2000, 3), dtype=torch.float32, device="cuda")
        o = dt.dtree_opts()
        o.bound = 3
        rc = dt._lib.dtree_knn(None, tr.handle, 3, ctypes.c_void_p(oi.data_ptr()),
                               ctypes.c_void_p(od.data_ptr()), ctypes.byref(o), None, None)
        assert rc == -1  # DTREE_ERR_INVALID_ARG
    finally:
        tr.free()
