"""Parity of the CUDA k-furthest-neighbour path (through the C ABI) with the
float64 oracle: every index and distance must match exactly."""
import functools

import numpy as np
import pytest
import torch

from oracle import kfn as okfn
from paper_1304_4327_gb300 import inputs
from test_oracle_kfn import load_figure1_kfn

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def dt():
    from paper_1304_4327_gb300 import build
    build.build()
    from paper_1304_4327_gb300 import dtree
    return dtree


def run(dt, ref, query, k, leaf=32, stats=False):
    tr = dt.dtree_build(torch.from_numpy(np.ascontiguousarray(ref, dtype=np.float32)).cuda(), leaf)
    tq = None if query is None else dt.dtree_build(
        torch.from_numpy(np.ascontiguousarray(query, dtype=np.float32)).cuda(), leaf)
    try:
        out = dt.dtree_kfn(tq, tr, k, with_stats=stats)
    finally:
        tr.free()
        if tq is not None:
            tq.free()
    res = (out[0].cpu().numpy(), out[1].cpu().numpy())
    return res + ((out[2],) if stats else ())


def check(dt, ref, query, k, leaf=32, truth=None):
    idx, dist, st = run(dt, ref, query, k, leaf, stats=True)
    ti, td = truth if truth is not None else okfn.kfn_brute(ref, query, k)
    ti, td = ti[:, :k], td[:, :k]  # (a longer exact list's prefix is the shorter one)
    assert np.array_equal(idx, ti), np.argwhere(idx != ti)[:5]
    assert np.array_equal(dist, np.sqrt(td).astype(np.float32))
    return st


@functools.lru_cache(maxsize=None)
def _gmm16(mono):
    W = inputs.gmm16(n_ref=12_000, n_query=3_000)
    query = None if mono else W.query
    return W, okfn.kfn_brute(W.ref, query, 63)


@pytest.mark.parametrize("k", [1, 2, 3, 4])
@pytest.mark.parametrize("leaf", [1, 2, 5])
def test_figure1(dt, k, leaf):
    P, I, D = load_figure1_kfn()
    idx, dist = run(dt, P, None, k, leaf)
    assert np.array_equal(idx, I[:, :k])
    assert np.array_equal(dist, np.sqrt(D[:, :k]).astype(np.float32))


@pytest.mark.parametrize("k", [1, 10, 63])
@pytest.mark.parametrize("mono", [False, True])
def test_gmm16(dt, k, mono):
    W, truth = _gmm16(mono)
    st = check(dt, W.ref, None if mono else W.query, k, truth=truth)
    nq = len(W.ref) if mono else len(W.query)
    # the inverted Score prunes: far fewer distances than all pairs
    assert 0 < st["point_pairs"] < 0.5 * nq * len(W.ref)
    assert st["node_pairs_pruned"] > 0


@pytest.mark.parametrize("d", [1, 2, 3, 5, 8, 13, 16, 33, 64])
def test_uniform_widths(dt, d):
    n = 6_000 if d <= 16 else 3_000
    R = inputs.uniform(n, d, 31 + d)
    Q = inputs.uniform(n // 4, d, 71 + d)
    check(dt, R, Q, 7, leaf=16)
    check(dt, R, None, 5, leaf=16)


def test_lattice_ties_take_the_float64_pass(dt):
    g = np.random.default_rng(3)
    R = g.integers(0, 4, size=(3_000, 3)).astype(np.float32)  # many exact duplicates
    st = check(dt, R, None, 12, leaf=8)
    assert st["fallback_queries"] > 0


def test_offset_cloud(dt):
    # large coordinates, small spread: keys near each other relative to their size
    g = np.random.default_rng(5)
    R = (1000.0 + g.normal(size=(5_000, 8))).astype(np.float32)
    Q = (1000.0 + g.normal(size=(800, 8))).astype(np.float32)
    check(dt, R, Q, 9)


@pytest.mark.parametrize("m,leaf,k", [(2, 1, 1), (3, 1, 2), (17, 2, 16), (100, 7, 63), (1000, 1024, 20)])
def test_tiny_and_ragged(dt, m, leaf, k):
    R = np.random.default_rng(m).normal(size=(m, 4)).astype(np.float32)
    check(dt, R, None, k, leaf)


def test_errors(dt):
    R = torch.from_numpy(inputs.uniform(1000, 3, 1)).cuda()
    tr = dt.dtree_build(R, 16)
    try:
        for k, status in ((0, -2), (1000, -2), (64, -7)):
            with pytest.raises(dt.DTreeError) as e:
                dt.dtree_kfn(None, tr, k)
            assert e.value.status == status, k
        with pytest.raises(dt.DTreeError) as e:
            dt.dtree_kfn(None, tr, 3, precision="bf16")
        assert e.value.status == -7
    finally:
        tr.free()
