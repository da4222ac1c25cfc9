"""Pins of the range-search oracle (no GPU): the paper's Figure 1 points with
hand-computed sets, closed forms on a line, invariants of the definition, the
dual-tree with the sound Score against brute force, and the printed Score
shown to lose results."""
import math
import os

import numpy as np
import pytest

from oracle import rangesearch as rs

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "figure1_range.txt")
RANGES = {"A": (0.5, math.sqrt(2.0)), "B": (2.0, math.sqrt(4.5))}


def load_figure1_range():
    pts, sets, mode = [], {}, None
    with open(GOLDEN) as f:
        for line in f:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            if line in ("points", "A", "B"):
                mode = line
                continue
            if mode == "points":
                pts.append([float(v) for v in line.split()])
            else:
                q, rest = line.split(":")
                rest = rest.strip()
                sets.setdefault(mode, {})[int(q)] = [] if rest == "-" else [int(v) for v in rest.split()]
    return np.array(pts, dtype=np.float32), sets


def segments(off, idx):
    return [list(idx[off[i]:off[i + 1]]) for i in range(len(off) - 1)]


@pytest.mark.parametrize("name", ["A", "B"])
def test_figure1_by_hand(name):
    P, sets = load_figure1_range()
    lo, hi = RANGES[name]
    off, idx, dist = rs.range_brute(P, None, lo, hi)
    assert segments(off, idx) == [sets[name][i] for i in range(5)]
    assert np.all((dist >= lo) & (dist <= hi))


@pytest.mark.parametrize("name", ["A", "B"])
@pytest.mark.parametrize("leaf", [1, 2, 3])
def test_figure1_dualtree(name, leaf):
    P, sets = load_figure1_range()
    lo, hi = RANGES[name]
    off, idx, _ = rs.range_dualtree(P, None, lo, hi, leaf_size=leaf)
    assert segments(off, idx) == [sets[name][i] for i in range(5)]


def test_points_on_a_line():
    # x_i = i: the neighbours of i in [1.5, 3] are i +- 2 and i +- 3 inside [0, m)
    m = 15
    P = np.zeros((m, 2), dtype=np.float32)
    P[:, 0] = np.arange(m)
    off, idx, dist = rs.range_brute(P, None, 1.5, 3.0)
    for i, seg in enumerate(segments(off, idx)):
        assert seg == sorted(j for j in (i - 3, i - 2, i + 2, i + 3) if 0 <= j < m), i
    assert np.all((dist == 2.0) | (dist == 3.0))


def test_definition_invariants():
    g = np.random.default_rng(4)
    R = g.normal(size=(200, 3)).astype(np.float32)
    # the whole line: every other point; mono symmetry
    off, idx, _ = rs.range_brute(R, None, 0.0, np.inf)
    assert all(seg == [j for j in range(200) if j != i] for i, seg in enumerate(segments(off, idx)))
    off, idx, _ = rs.range_brute(R, None, 0.7, 1.9)
    pairs = {(i, j) for i, seg in enumerate(segments(off, idx)) for j in seg}
    assert pairs and all((j, i) in pairs for i, j in pairs)
    # two adjacent ranges split one range (they share only the exact boundary)
    Q = g.normal(size=(30, 3)).astype(np.float32)
    a = segments(*rs.range_brute(R, Q, 0.5, 1.0)[:2])
    b = segments(*rs.range_brute(R, Q, np.nextafter(1.0, 2.0), 2.0)[:2])
    c = segments(*rs.range_brute(R, Q, 0.5, 2.0)[:2])
    assert all(sorted(x + y) == z for x, y, z in zip(a, b, c))


@pytest.mark.parametrize("seed", range(6))
def test_dualtree_matches_brute_force(seed):
    g = np.random.default_rng(200 + seed)
    n, d = int(g.integers(20, 150)), int(g.integers(1, 5))
    R = (g.integers(0, 5, size=(n, d)) if seed % 2 else g.normal(size=(n, d))).astype(np.float32)
    lo, hi = sorted(g.uniform(0.0, 3.0, size=2))
    for query in (None, g.normal(size=(25, d)).astype(np.float32)):
        bo, bi, bd = rs.range_brute(R, query, lo, hi)
        to, ti, td = rs.range_dualtree(R, query, lo, hi, leaf_size=int(g.integers(1, 6)))
        assert np.array_equal(bo, to) and np.array_equal(bi, ti) and np.array_equal(bd, td)


def test_sound_score_prunes():
    g = np.random.default_rng(9)
    R = np.concatenate([g.normal(size=(100, 2)), 40 + g.normal(size=(100, 2))]).astype(np.float32)
    st = {}
    rs.range_dualtree(R, None, 0.0, 1.0, leaf_size=4, stats=st)
    assert st["prunes"] > 0 and st["basecases"] < 0.5 * 200 * 199


def test_printed_score_loses_results():
    # the printed Score also prunes pairs with d_min < delta1 <= d_max
    g = np.random.default_rng(1)
    R = g.normal(size=(120, 2)).astype(np.float32)
    bo, bi, _ = rs.range_brute(R, None, 1.0, 2.0)
    lo_, li_, _ = rs.range_dualtree(R, None, 1.0, 2.0, leaf_size=4, literal=True)
    assert len(li_) < len(bi)
    so, si, _ = rs.range_dualtree(R, None, 1.0, 2.0, leaf_size=4)
    assert np.array_equal(si, bi) and np.array_equal(so, bo)
