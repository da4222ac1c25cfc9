"""Pins of the k-furthest-neighbour oracle (no GPU): the paper's Figure 1
points with hand-computed lists, closed forms on a line, invariants of the
definition, and the inverted dual-tree of Section 5 against brute force."""
import os

import numpy as np
import pytest

from oracle import kfn

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "figure1_kfn.txt")


def load_figure1_kfn():
    pts, lists, mode = [], {}, None
    with open(GOLDEN) as f:
        for line in f:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            if line in ("points", "lists"):
                mode = line
                continue
            if mode == "points":
                pts.append([float(v) for v in line.split()])
            else:
                q, rest = line.split(":")
                idx, d2 = rest.split("|")
                lists[int(q)] = ([int(v) for v in idx.split()], [float(v) for v in d2.split()])
    P = np.array(pts, dtype=np.float32)
    I = np.array([lists[i][0] for i in range(len(pts))], dtype=np.int64)
    D = np.array([lists[i][1] for i in range(len(pts))], dtype=np.float64)
    return P, I, D


@pytest.mark.parametrize("k", [1, 2, 3, 4])
def test_figure1_by_hand(k):
    P, I, D = load_figure1_kfn()
    idx, d2 = kfn.kfn_brute(P, None, k)
    assert np.array_equal(idx, I[:, :k])
    assert np.array_equal(d2, D[:, :k])


@pytest.mark.parametrize("k", [1, 2, 3, 4])
@pytest.mark.parametrize("leaf", [1, 2, 3])
def test_figure1_dualtree(k, leaf):
    P, I, D = load_figure1_kfn()
    idx, d2 = kfn.kfn_dualtree(P, None, k, leaf_size=leaf)
    assert np.array_equal(idx, I[:, :k]) and np.array_equal(d2, D[:, :k])


def test_points_on_a_line():
    # x_i = i on the first axis: the furthest point is the farther end, and
    # the query midway sees both ends at once (the lower index, 0, first)
    m = 21
    P = np.zeros((m, 3), dtype=np.float32)
    P[:, 0] = np.arange(m)
    idx, d2 = kfn.kfn_brute(P, None, 1)
    for i in range(m):
        assert idx[i, 0] == (0 if i >= (m - 1) / 2 else m - 1), i
        assert d2[i, 0] == max(i, m - 1 - i) ** 2
    mid = (m - 1) // 2
    idx, d2 = kfn.kfn_brute(P, None, 4)
    assert list(idx[mid]) == [0, m - 1, 1, m - 2]
    assert list(d2[mid]) == [mid ** 2, mid ** 2, (mid - 1) ** 2, (mid - 1) ** 2]
    # an external query beyond the right end: the order is simply by position
    q = np.array([[40.0, 0.0, 0.0]], dtype=np.float32)
    idx, d2 = kfn.kfn_brute(P, q, m)
    assert list(idx[0]) == list(range(m))
    assert np.array_equal(d2[0], (40.0 - np.arange(m)) ** 2)


def test_definition_invariants():
    g = np.random.default_rng(11)
    R = g.normal(size=(300, 5)).astype(np.float32)
    Q = g.normal(size=(40, 5)).astype(np.float32)
    idx, d2 = kfn.kfn_brute(R, Q, 300)
    full = ((Q[:, None, :].astype(np.float64) - R[None, :, :].astype(np.float64)) ** 2).sum(-1)
    assert np.all(np.diff(d2, axis=1) <= 0)                      # descending
    assert np.allclose(d2[:, 0], full.max(axis=1), rtol=1e-12)   # the maximum first
    assert all(sorted(r) == list(range(300)) for r in idx)       # k = m: every point once
    # monochromatic: never the query itself, and m - 1 entries are all the others
    idx, _ = kfn.kfn_brute(R, None, 299)
    assert all(i not in row for i, row in enumerate(idx))


@pytest.mark.parametrize("seed", range(6))
def test_dualtree_matches_brute_force(seed):
    g = np.random.default_rng(100 + seed)
    n, d = int(g.integers(20, 160)), int(g.integers(1, 6))
    kind = seed % 3
    if kind == 0:
        R = g.normal(size=(n, d))
    elif kind == 1:  # two clusters far apart
        R = np.concatenate([g.normal(size=(n // 2, d)), 30 + g.normal(size=(n - n // 2, d))])
    else:  # an integer lattice: many exact ties
        R = g.integers(0, 4, size=(n, d)).astype(np.float64)
    R = R.astype(np.float32)
    k = int(g.integers(1, min(12, n - 1)))
    leaf = int(g.integers(1, 8))
    st = {}
    for query in (None, g.normal(size=(30, d)).astype(np.float32)):
        bi, bd = kfn.kfn_brute(R, query, k)
        ti, td = kfn.kfn_dualtree(R, query, k, leaf_size=leaf, stats=st)
        assert np.array_equal(bi, ti) and np.array_equal(bd, td)


def test_dualtree_prunes():
    g = np.random.default_rng(7)
    R = np.concatenate([g.normal(size=(150, 3)), 50 + g.normal(size=(150, 3))]).astype(np.float32)
    st = {}
    kfn.kfn_dualtree(R, None, 5, leaf_size=8, stats=st)
    assert st["prunes"] > 0
    assert st["basecases"] < 0.8 * 300 * 299


def test_pruning_at_equality_loses_ties():
    # the planted mistake: pruning when d_max == B' drops equal-distance,
    # lower-index points on a lattice, where exact ties abound
    failures = 0
    for seed in range(40):
        g = np.random.default_rng(seed)
        R = g.integers(0, 3, size=(60, 2)).astype(np.float32)
        bi, bd = kfn.kfn_brute(R, None, 3)
        ti, td = kfn.kfn_dualtree(R, None, 3, leaf_size=2, strict=False)
        failures += not np.array_equal(bi, ti)
        # the sound (strict) traversal agrees on the same inputs
        si, sd = kfn.kfn_dualtree(R, None, 3, leaf_size=2)
        assert np.array_equal(bi, si) and np.array_equal(bd, sd)
    assert failures > 0
