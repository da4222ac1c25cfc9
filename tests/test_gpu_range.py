"""Parity of the CUDA range search (through the C ABI) with the float64
oracle: every query's set of neighbours and their distances must match
exactly (the sets are compared in index order)."""
import functools
import math

import numpy as np
import pytest
import torch

from oracle import rangesearch as ors
from paper_1304_4327_gb300 import inputs
from test_oracle_range import RANGES, load_figure1_range

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def dt():
    from paper_1304_4327_gb300 import build
    build.build()
    from paper_1304_4327_gb300 import dtree
    return dtree


def run(dt, ref, query, lo, hi, leaf=32):
    tr = dt.dtree_build(torch.from_numpy(np.ascontiguousarray(ref, dtype=np.float32)).cuda(), leaf)
    tq = None if query is None else dt.dtree_build(
        torch.from_numpy(np.ascontiguousarray(query, dtype=np.float32)).cuda(), leaf)
    try:
        off, idx, dist, st = dt.dtree_range(tq, tr, lo, hi, with_stats=True)
    finally:
        tr.free()
        if tq is not None:
            tq.free()
    return off.cpu().numpy(), idx.cpu().numpy(), dist.cpu().numpy(), st


def check(dt, ref, query, lo, hi, leaf=32):
    off, idx, dist, st = run(dt, ref, query, lo, hi, leaf)
    to, ti, td = ors.range_brute(ref, query, lo, hi)
    assert np.array_equal(off, to)
    for i in range(len(off) - 1):
        s = slice(off[i], off[i + 1])
        order = np.argsort(idx[s], kind="stable")
        assert np.array_equal(idx[s][order], ti[s]), i
        assert np.array_equal(dist[s][order], td[s].astype(np.float32)), i
    return st


@pytest.mark.parametrize("name", ["A", "B"])
@pytest.mark.parametrize("leaf", [1, 2, 5])
def test_figure1(dt, name, leaf):
    P, sets = load_figure1_range()
    lo, hi = RANGES[name]
    off, idx, _, _ = run(dt, P, None, lo, hi, leaf)
    for i in range(5):
        assert sorted(idx[off[i]:off[i + 1]]) == sets[name][i]


@functools.lru_cache(maxsize=None)
def _gmm():
    return inputs.gmm16(n_ref=8_000, n_query=2_000)


@pytest.mark.parametrize("lo,hi", [(0.0, 2.5), (2.0, 3.0), (10.0, 11.0), (0.0, 0.0)])
@pytest.mark.parametrize("mono", [False, True])
def test_gmm16(dt, lo, hi, mono):
    W = _gmm()
    st = check(dt, W.ref, None if mono else W.query, lo, hi)
    nq = len(W.ref) if mono else len(W.query)
    if hi < 5:
        assert st["point_pairs"] < 0.5 * nq * len(W.ref)  # the Score prunes


@pytest.mark.parametrize("d", [1, 2, 3, 8, 16, 33, 64])
def test_uniform_widths(dt, d):
    n = 4_000 if d <= 16 else 2_000
    R = inputs.uniform(n, d, 40 + d)
    Q = inputs.uniform(n // 4, d, 80 + d)
    r = 0.3 * math.sqrt(d)  # about the typical spacing
    check(dt, R, Q, 0.5 * r, r, leaf=16)
    check(dt, R, None, 0.0, r, leaf=16)


def test_lattice_boundaries_are_inclusive(dt):
    # integer points: many distances fall exactly on the ends sqrt(2) and 2
    g = np.random.default_rng(2)
    R = g.integers(0, 6, size=(2_500, 2)).astype(np.float32)
    st = check(dt, R, None, math.sqrt(2.0), 2.0, leaf=8)
    assert st["rerank_candidates"] > 0  # the boundary cases were decided in float64


def test_whole_and_empty_ranges(dt):
    R = np.random.default_rng(8).normal(size=(500, 3)).astype(np.float32)
    off, idx, _, _ = run(dt, R, None, 0.0, math.inf)
    assert off[-1] == 500 * 499
    off, idx, dist, _ = run(dt, R, None, 1e6, 2e6)
    assert off[-1] == 0 and len(idx) == 0 and len(dist) == 0


def test_errors(dt):
    R = torch.from_numpy(inputs.uniform(1000, 3, 1)).cuda()
    tr = dt.dtree_build(R, 16)
    try:
        for lo, hi in ((-1.0, 1.0), (2.0, 1.0), (math.nan, 1.0), (0.0, math.nan)):
            with pytest.raises(dt.DTreeError) as e:
                dt.dtree_range(None, tr, lo, hi)
            assert e.value.status == -1, (lo, hi)
        with pytest.raises(dt.DTreeError) as e:
            dt.dtree_range(None, tr, 0.0, 1.0, precision="tf32")
        assert e.value.status == -7
    finally:
        tr.free()
