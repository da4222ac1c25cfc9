"""The per-query cap pass: a budgeted best-first search that bounds each
query's k-th distance before the traversal.  It only tightens B(N_q) and the
BaseCase's insertion threshold, so every budget (and no cap pass at all)
must give the oracle's answer, bit for bit the same."""
import functools

import numpy as np
import pytest
import torch

from paper_1304_4327_gb300 import inputs
from parity import compare
from test_gpu_knn import truth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def dt():
    from paper_1304_4327_gb300 import build
    build.build()
    from paper_1304_4327_gb300 import dtree
    return dtree


def _trees(dt, ref, query, leaf=32):
    tr = dt.dtree_build(torch.from_numpy(np.ascontiguousarray(ref)).cuda(), leaf)
    tq = None if query is None else dt.dtree_build(torch.from_numpy(np.ascontiguousarray(query)).cuda(), leaf)
    return tr, tq


@functools.lru_cache(maxsize=None)
def _workload():
    return inputs.gmm16(n_ref=20_000, n_query=5_000)


@functools.lru_cache(maxsize=None)
def _truth(mono, k):
    W = _workload()
    return truth(W.ref, None if mono else W.query, k)


@pytest.mark.parametrize("precision", ["fp32", "tf32", "bf16"])
@pytest.mark.parametrize("mono", [False, True])
@pytest.mark.parametrize("k", [1, 10, 31])
def test_every_budget_gives_the_same_exact_answer(dt, precision, mono, k):
    W = _workload()
    query = None if mono else W.query
    tr, tq = _trees(dt, W.ref, query)
    try:
        outs = {}
        for cap in (-1, 1, 3, 8, 17):
            idx, dist, st = dt.dtree_knn(tq, tr, k, precision=precision, with_stats=True,
                                         cap_leaves=cap)
            outs[cap] = (idx.cpu().numpy(), dist.cpu().numpy(), st)
        ti, td = _truth(mono, k)
        compare(outs[8][0], outs[8][1], ti, td, k)
        for cap, (i, d, _) in outs.items():
            assert np.array_equal(i, outs[-1][0]) and np.array_equal(d, outs[-1][1]), cap
        # the cap tightens B(N_q): the traversal emits no more leaf pairs
        assert outs[8][2]["leaf_pairs_emitted"] <= outs[-1][2]["leaf_pairs_emitted"]
    finally:
        tr.free()
        if tq is not None:
            tq.free()


def test_cap_prunes_on_clustered_data(dt):
    W = inputs.gmm16(n_ref=200_000, n_query=50_000)
    tr, tq = _trees(dt, W.ref, W.query)
    try:
        _, _, off = dt.dtree_knn(tq, tr, 10, precision="bf16", with_stats=True, cap_leaves=-1)
        _, _, on = dt.dtree_knn(tq, tr, 10, precision="bf16", with_stats=True, cap_leaves=8)
        print("leaf pairs without / with the cap:", off["leaf_pairs_emitted"], on["leaf_pairs_emitted"])
        assert on["leaf_pairs_emitted"] < 0.9 * off["leaf_pairs_emitted"]
    finally:
        tr.free()
        tq.free()


def test_tiny_trees_and_ragged_leaves(dt):
    # fewer points than a budget's leaves, leaves of one and two points, k up
    # to m - 1 (and up to the float32 lists' 63)
    g = np.random.default_rng(5)
    for m, leaf, k in ((3, 1, 2), (17, 2, 16), (100, 7, 63)):
        R = g.normal(size=(m, 5)).astype(np.float32)
        tr, _ = _trees(dt, R, None, leaf)
        try:
            for cap in (-1, 17):
                idx, dist = dt.dtree_knn(None, tr, k, cap_leaves=cap)
                ti, td = truth(R, None, k)
                compare(idx.cpu().numpy(), dist.cpu().numpy(), ti, td, k)
        finally:
            tr.free()


@pytest.mark.parametrize("cap", [-2, 18])
def test_budget_out_of_range_is_rejected(dt, cap):
    tr, _ = _trees(dt, inputs.uniform(2000, 4, 3), None, 16)
    try:
        with pytest.raises(dt.DTreeError) as e:
            dt.dtree_knn(None, tr, 3, cap_leaves=cap)
        assert e.value.status == -1
    finally:
        tr.free()
