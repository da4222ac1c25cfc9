"""Pins of the minimum-spanning-tree oracle (no GPU): Kruskal against Prim
(two algorithms for the same unique tree), closed forms, and the tree
properties that any minimum spanning tree has."""
import numpy as np
import pytest

from oracle import emst


def test_points_on_a_line():
    # x_i = i (shuffled order): consecutive points, total length m - 1
    g = np.random.default_rng(0)
    m = 30
    pos = g.permutation(m)
    P = np.zeros((m, 3), dtype=np.float32)
    P[:, 0] = pos
    e, d2 = emst.emst_kruskal(P)
    assert len(e) == m - 1 and np.all(d2 == 1.0)
    assert sorted(tuple(sorted((pos[a], pos[b]))) for a, b in e) == [(i, i + 1) for i in range(m - 1)]


def test_unit_square_ties():
    # four corners: the three sides of smallest (lo, hi) win among equal lengths
    P = np.array([[0, 0], [1, 0], [1, 1], [0, 1]], dtype=np.float32)
    e, d2 = emst.canonical(*emst.emst_kruskal(P))
    assert e.tolist() == [[0, 1], [0, 3], [1, 2]] and np.all(d2 == 1.0)
    e2, _ = emst.canonical(*emst.emst_prim(P))
    assert e2.tolist() == e.tolist()


@pytest.mark.parametrize("seed", range(8))
def test_kruskal_equals_prim(seed):
    g = np.random.default_rng(50 + seed)
    n, d = int(g.integers(2, 300)), int(g.integers(1, 6))
    kind = seed % 3
    if kind == 0:
        P = g.normal(size=(n, d))
    elif kind == 1:  # clusters far apart
        P = g.normal(size=(n, d)) + 40 * g.integers(0, 3, size=(n, 1))
    else:  # a lattice with duplicates: many equal weights
        P = g.integers(0, 4, size=(n, d))
    P = P.astype(np.float32)
    ek, wk = emst.canonical(*emst.emst_kruskal(P))
    ep, wp = emst.canonical(*emst.emst_prim(P))
    assert np.array_equal(ek, ep) and np.array_equal(wk, wp)


def test_tree_properties():
    g = np.random.default_rng(3)
    P = g.normal(size=(150, 3)).astype(np.float32)
    e, d2 = emst.emst_kruskal(P)
    n = len(P)
    # n - 1 edges that connect every point
    parent = list(range(n))

    def find(a):
        while parent[a] != a:
            a = parent[a]
        return a
    for a, b in e:
        parent[find(a)] = find(b)
    assert len(e) == n - 1 and len({find(i) for i in range(n)}) == 1
    # the cycle property: a non-tree edge weighs at least every tree edge on
    # the tree path between its ends
    adj = {i: [] for i in range(n)}
    for (a, b), w in zip(e, d2):
        adj[a].append((b, w))
        adj[b].append((a, w))

    def path_max(s, t):
        stack, seen = [(s, 0.0)], {s}
        while stack:
            u, mx = stack.pop()
            if u == t:
                return mx
            for v, w in adj[u]:
                if v not in seen:
                    seen.add(v)
                    stack.append((v, max(mx, w)))
    X = P.astype(np.float64)
    tree = {tuple(x) for x in e.tolist()}
    for _ in range(200):
        a, b = sorted(g.choice(n, 2, replace=False))
        if (a, b) in tree:
            continue
        w = float(((X[a] - X[b]) ** 2).sum())
        assert w >= path_max(a, b) - 1e-12


def test_a_wrong_tie_order_changes_the_tree():
    # the planted mistake: ordering equal weights by the higher index first
    # picks other edges on a lattice, so the tie rule is part of the pin
    P = np.array([[0, 0], [1, 0], [1, 1], [0, 1]], dtype=np.float32)
    e, _ = emst.canonical(*emst.emst_kruskal(P))
    assert [0, 3] in e.tolist() and [2, 3] not in e.tolist()
