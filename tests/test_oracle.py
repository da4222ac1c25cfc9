"""Pins for the CPU oracle (runs without a GPU).

The oracle is checked against facts that do not come from itself: the paper's
Figure 1 worked example (hand-computed lists), closed forms on integer
lattices, an independent library kd-tree (scipy.spatial.cKDTree), the
paper's correctness argument (a non-pruning traversal equals brute force; the
bound never prunes a true neighbour), and recorded counterexamples for the two
printed formulas that the oracle reads differently.
"""
import os

import numpy as np
import pytest

import oracle
from paper_1304_4327_gb300 import inputs

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "figure1_knn.txt")


def load_figure1():
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


# --------------------------------------------------------------------------
# Figure 1 worked example
# --------------------------------------------------------------------------

@pytest.mark.parametrize("k", [1, 2, 3, 4])
def test_figure1_brute(k):
    P, I, D = load_figure1()
    idx, d2 = oracle.knn_brute(P, None, k)
    assert np.array_equal(idx, I[:, :k])
    assert np.array_equal(d2, D[:, :k])


@pytest.mark.parametrize("k", [1, 2, 3, 4])
@pytest.mark.parametrize("leaf", [1, 2, 5])
@pytest.mark.parametrize("bound", [oracle.BOUND_SOUND, oracle.BOUND_B1, oracle.BOUND_NONE])
def test_figure1_dualtree(k, leaf, bound):
    P, I, D = load_figure1()
    idx, d2, st = oracle.knn_dualtree(P, None, k, leaf, bound)
    assert np.array_equal(idx, I[:, :k])
    assert np.array_equal(d2, D[:, :k])


def test_figure1_exact_tie_at_k2():
    # row 4 sees rows 0 and 3 at exactly sqrt(0.5): the lower index wins the k=2 slot
    P, _, _ = load_figure1()
    idx, d2 = oracle.knn_brute(P, None, 2)
    assert idx[4].tolist() == [1, 0]
    assert d2[4, 1] == 0.5


@pytest.mark.parametrize("leaf", [1, 2, 5])
def test_figure1_gray_allnn(leaf):
    P, I, D = load_figure1()
    idx, d2 = oracle.allnn_gray(P, None, leaf)
    assert np.array_equal(idx, I[:, 0])
    assert np.array_equal(d2, D[:, 0])


# --------------------------------------------------------------------------
# closed forms on integer lattices
# --------------------------------------------------------------------------

def lattice1d_expected(n, k):
    # neighbours of i on {0..n-1}: distance 1, 2, ... ; at equal distance the
    # lower index (i - t) comes before (i + t)
    out = []
    for i in range(n):
        lst = []
        t = 1
        while len(lst) < k:
            for j in (i - t, i + t):
                if 0 <= j < n and len(lst) < k:
                    lst.append(j)
            t += 1
        out.append(lst)
    return np.array(out, dtype=np.int64)


@pytest.mark.parametrize("k", [1, 2, 3, 6])
def test_lattice_1d(k):
    n = 40
    X = inputs.lattice([n])
    exp = lattice1d_expected(n, k)
    idx, d2 = oracle.knn_brute(X, None, k)
    assert np.array_equal(idx, exp)
    assert np.array_equal(d2, (exp - np.arange(n)[:, None]).astype(np.float64) ** 2)
    idx2, _, _ = oracle.knn_dualtree(X, None, k, 3)
    assert np.array_equal(idx2, exp)


def test_lattice_2d_interior():
    # 7x7 grid, row-major index x*7+y; an interior point's four unit
    # neighbours in index order are i-7, i-1, i+1, i+7; the next four (at
    # sqrt 2) are i-8, i-6, i+6, i+8
    X = inputs.lattice([7, 7])
    idx, d2 = oracle.knn_brute(X, None, 8)
    for x in range(1, 6):
        for y in range(1, 6):
            i = x * 7 + y
            assert idx[i].tolist() == [i - 7, i - 1, i + 1, i + 7, i - 8, i - 6, i + 6, i + 8]
            assert d2[i].tolist() == [1, 1, 1, 1, 2, 2, 2, 2]
    idx2, d22, _ = oracle.knn_dualtree(X, None, 8, 4)
    assert np.array_equal(idx2, idx) and np.array_equal(d22, d2)


# --------------------------------------------------------------------------
# an independent library kd-tree
# --------------------------------------------------------------------------

@pytest.mark.parametrize("d", [2, 3, 8, 16])
@pytest.mark.parametrize("k", [1, 5, 10])
def test_brute_vs_scipy(d, k):
    ckd = pytest.importorskip("scipy.spatial").cKDTree
    R = inputs.gaussian(2000, d, 100 + d)
    Q = inputs.uniform(300, d, 200 + d)
    idx, d2 = oracle.knn_brute(R, Q, k)
    sd, si = ckd(R.astype(np.float64)).query(Q.astype(np.float64), k)
    si = si.reshape(len(Q), k)
    sd = sd.reshape(len(Q), k)
    assert np.array_equal(idx, si)
    np.testing.assert_allclose(np.sqrt(d2), sd, rtol=1e-12, atol=0)


def test_mono_vs_scipy():
    ckd = pytest.importorskip("scipy.spatial").cKDTree
    X = inputs.uniform(1500, 3, 7)
    idx, d2 = oracle.knn_brute(X, None, 5)
    sd, si = ckd(X.astype(np.float64)).query(X.astype(np.float64), 6)
    assert np.array_equal(si[:, 0], np.arange(len(X)))       # no duplicates: self first
    assert np.array_equal(idx, si[:, 1:])


# --------------------------------------------------------------------------
# the correctness argument: traversal == brute force, bound is safe
# --------------------------------------------------------------------------

DATA = {
    "uniform": lambda n, d, s: inputs.uniform(n, d, s),
    "gaussian": lambda n, d, s: inputs.gaussian(n, d, s),
    "duplicates": lambda n, d, s: inputs.duplicate_heavy(n, d, s),
    "collinear": lambda n, d, s: inputs.collinear(n, d, s),
}


@pytest.mark.parametrize("kind", sorted(DATA))
@pytest.mark.parametrize("d", [1, 3, 8, 16])
@pytest.mark.parametrize("mono", [True, False])
def test_dualtree_equals_brute(kind, d, mono):
    R = DATA[kind](500, d, 1000 + d)
    Q = None if mono else DATA[kind](200, d, 2000 + d)
    for k in (1, 5, 10):
        truth = oracle.knn_brute(R, Q, k)
        for leaf in (1, 5, 20):
            for bound in (oracle.BOUND_SOUND, oracle.BOUND_B1, oracle.BOUND_NONE):
                idx, d2, st = oracle.knn_dualtree(R, Q, k, leaf, bound, truth=truth)
                assert np.array_equal(idx, truth[0]), (k, leaf, bound)
                assert np.array_equal(d2, truth[1])
                assert st["audit_prune"] == 0 and st["audit_bound"] == 0
                assert st["order"] == 0 and st["incomplete"] == 0


def test_dualtree_prunes_and_audits_clean():
    W = inputs.mono_uniform()
    truth = oracle.knn_brute(W.ref, None, W.k)
    idx, d2, st = oracle.knn_dualtree(W.ref, None, W.k, W.leaf_size, truth=truth)
    assert np.array_equal(idx, truth[0])
    n = len(W.ref)
    assert st["prunes"] > 0 and st["basecases"] < n * (n - 1) // 2
    assert st["audit_prune"] == 0 and st["audit_bound"] == 0


def test_no_prune_traversal_visits_every_pair():
    X = inputs.uniform(300, 2, 5)
    _, _, st = oracle.knn_dualtree(X, None, 3, 4, oracle.BOUND_NONE)
    assert st["prunes"] == 0
    assert st["basecases"] == 300 * 299


@pytest.mark.parametrize("par_depth", [1, 3, 5])
def test_parallel_subtrees_equal_serial(par_depth):
    R = inputs.gaussian(4000, 3, 31)
    Q = inputs.gaussian(1500, 3, 32)
    truth = oracle.knn_brute(R, Q, 7)
    idx, d2, st = oracle.knn_dualtree(R, Q, 7, 16, par_depth=par_depth, truth=truth)
    assert np.array_equal(idx, truth[0]) and np.array_equal(d2, truth[1])
    assert st["audit_prune"] == 0


def test_literal_combined_bound_is_unsound():
    # The combined recursion exactly as printed in Section 5 uses
    # B(N_c) + 2(lambda_q - lambda_c) for every child, although that step was
    # derived for B_2 only.  On this 6-point input it prunes a true neighbour.
    X = inputs.uniform(6, 2, 13)
    truth = oracle.knn_brute(X, None, 1)
    idx, _, st = oracle.knn_dualtree(X, None, 1, 1, oracle.BOUND_LITERAL, truth=truth)
    assert st["audit_bound"] > 0 and st["audit_prune"] > 0
    assert not np.array_equal(idx, truth[0])
    idx_s, _, st_s = oracle.knn_dualtree(X, None, 1, 1, oracle.BOUND_SOUND, truth=truth)
    assert np.array_equal(idx_s, truth[0]) and st_s["audit_bound"] == 0


def test_gray_allnn_reading():
    # Algorithm 4's bound must equal B_1 (max over the node's points); the
    # printed per-pair line "if d < delta then delta = d" gives a wrong answer
    # on this 5-point input, the reading does not.
    X = inputs.uniform(5, 2, 1)
    truth = oracle.knn_brute(X, None, 1)
    gi, gd = oracle.allnn_gray(X, None, 3, variant=0)
    assert np.array_equal(gi, truth[0][:, 0]) and np.array_equal(gd, truth[1][:, 0])
    gi1, _ = oracle.allnn_gray(X, None, 3, variant=1)
    assert not np.array_equal(gi1, truth[0][:, 0])


@pytest.mark.parametrize("mono", [True, False])
def test_gray_allnn_equals_dualtree_k1(mono):
    R = inputs.gaussian(1200, 3, 41)
    Q = None if mono else inputs.uniform(500, 3, 42)
    gi, gd = oracle.allnn_gray(R, Q, 8)
    di, dd, _ = oracle.knn_dualtree(R, Q, 1, 8)
    assert np.array_equal(gi, di[:, 0]) and np.array_equal(gd, dd[:, 0])


# --------------------------------------------------------------------------
# problem-statement invariants and edge cases
# --------------------------------------------------------------------------

def test_self_exclusion_by_index_with_duplicates():
    # duplicates at distance 0 with other indices are valid neighbours
    X = np.array([[0, 0], [0, 0], [0, 0], [5, 5]], dtype=np.float32)
    idx, d2 = oracle.knn_brute(X, None, 2)
    assert idx.tolist() == [[1, 2], [0, 2], [0, 1], [0, 1]]
    assert d2[:3].tolist() == [[0, 0]] * 3
    idx2, d22, _ = oracle.knn_dualtree(X, None, 2, 1)
    assert np.array_equal(idx2, idx) and np.array_equal(d22, d2)


def test_k_range():
    X = inputs.uniform(10, 2, 3)
    idx, _ = oracle.knn_brute(X, None, 9)                     # k = m - 1 (mono)
    for i in range(10):
        assert sorted(idx[i].tolist()) == [j for j in range(10) if j != i]
    with pytest.raises(ValueError):
        oracle.knn_dualtree(X, None, 10, 2)                   # k > m - 1 (mono)
    idx, _ = oracle.knn_brute(X, X[:3], 10)                   # bichromatic k = m ...
    with pytest.raises(ValueError):
        oracle.knn_brute(X, X[:3], 11)                        # ... k > m has no answer


def test_outputs_ascending():
    R = inputs.gaussian(800, 4, 51)
    Q = inputs.gaussian(100, 4, 52)
    idx, d2, _ = oracle.knn_dualtree(R, Q, 10, 8)
    assert np.all(np.diff(d2, axis=1) >= 0)
    ties = np.diff(d2, axis=1) == 0
    assert np.all(np.diff(idx, axis=1)[ties] > 0)


def test_single_leaf_and_single_query():
    R = inputs.uniform(50, 3, 61)
    Q = inputs.uniform(1, 3, 62)
    truth = oracle.knn_brute(R, Q, 4)
    idx, d2, _ = oracle.knn_dualtree(R, Q, 4, 1000)
    assert np.array_equal(idx, truth[0])


@pytest.mark.parametrize("leaf", [1, 7, 32])
def test_kdtree_structure(leaf):
    X = inputs.gaussian(1000, 5, 71)
    nodes, leaves, depth, bad = oracle.kdtree_check(X, leaf)
    assert bad == 0
    assert nodes == 2 * leaves - 1
    assert depth >= int(np.ceil(np.log2(1000 / leaf))) - 1


# --------------------------------------------------------------------------
# Score's d_min as balls (a ball tree over the same splits) or as the larger
# of boxes and balls: the traversal stays exact and prunes no true neighbour
# --------------------------------------------------------------------------

@pytest.mark.parametrize("dmin", ["ball", "both"])
@pytest.mark.parametrize("k", [1, 2, 3, 4])
def test_figure1_dualtree_ball_bounds(dmin, k):
    P, I, D = load_figure1()
    for leaf in (1, 2, 5):
        idx, d2, st = oracle.knn_dualtree(P, None, k, leaf, dmin=dmin)
        assert np.array_equal(idx, I[:, :k])
        assert np.array_equal(d2, D[:, :k])


@pytest.mark.parametrize("dmin", ["ball", "both"])
@pytest.mark.parametrize("kind", sorted(DATA))
@pytest.mark.parametrize("d", [2, 8])
@pytest.mark.parametrize("mono", [True, False])
def test_dualtree_ball_bounds_equal_brute(dmin, kind, d, mono):
    R = DATA[kind](500, d, 3000 + d)
    Q = None if mono else DATA[kind](200, d, 4000 + d)
    for k in (1, 5):
        truth = oracle.knn_brute(R, Q, k)
        for leaf in (1, 8):
            idx, d2, st = oracle.knn_dualtree(R, Q, k, leaf, truth=truth, dmin=dmin)
            assert np.array_equal(idx, truth[0]), (k, leaf)
            assert np.array_equal(d2, truth[1])
            assert st["audit_prune"] == 0 and st["audit_bound"] == 0
            assert st["incomplete"] == 0


def test_ball_bound_prunes_separated_clusters():
    # two clusters 100 apart: every cross pair of leaves is far beyond both
    # balls' radii, so the ball bound alone prunes them
    g = np.random.default_rng(7)
    A = g.normal(0.0, 1.0, (300, 3))
    B = g.normal(0.0, 1.0, (300, 3)) + np.array([100.0, 0.0, 0.0])
    X = np.vstack([A, B]).astype(np.float32)
    truth = oracle.knn_brute(X, None, 3)
    idx, _, st = oracle.knn_dualtree(X, None, 3, 10, truth=truth, dmin="ball")
    assert np.array_equal(idx, truth[0])
    assert st["prunes"] > 0 and st["audit_prune"] == 0
    assert st["basecases"] < 600 * 599 // 2


def test_ball_bound_is_the_centre_distance_less_both_radii():
    # one leaf per tree side: two points each, so lambda is half the pair's
    # box diagonal and the ball distance has a closed form; a query cluster
    # whose k-th distance is smaller than that distance is pruned against it
    Q = np.array([[0.0, 0.0], [0.0, 1.0]], dtype=np.float32)
    R = np.array([[0.0, 0.0], [0.0, 1.0], [10.0, 0.0], [10.0, 1.0]], dtype=np.float32)
    # reference leaves {0, 1} and {2, 3}: centres (0, 0.5) and (10, 0.5),
    # lambda 0.5 each; the query leaf's centre (0, 0.5), lambda 0.5:
    # d_ball = 10 - 0.5 - 0.5 = 9 > B = 0 (k = 1, the query's own point)
    idx, d2, st = oracle.knn_dualtree(R, Q, 1, 2, dmin="ball")
    assert np.array_equal(idx[:, 0], [0, 1]) and np.array_equal(d2[:, 0], [0.0, 0.0])
    assert st["prunes"] >= 1 and st["basecases"] == 4
