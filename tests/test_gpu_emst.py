"""Parity of the CUDA minimum spanning tree (through the C ABI) with the
float64 oracle: the unique tree under the edge order, edge for edge."""
import numpy as np
import pytest
import torch

from oracle import emst as oemst
from paper_1304_4327_gb300 import inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def dt():
    from paper_1304_4327_gb300 import build
    build.build()
    from paper_1304_4327_gb300 import dtree
    return dtree


def run(dt, P, leaf=32):
    t = dt.dtree_build(torch.from_numpy(np.ascontiguousarray(P, dtype=np.float32)).cuda(), leaf)
    try:
        e, d, st = dt.dtree_emst(t, with_stats=True)
        e2, d2 = dt.dtree_emst(t)
        assert torch.equal(e, e2) and torch.equal(d, d2)  # the same order every call
    finally:
        t.free()
    return e.cpu().numpy(), d.cpu().numpy(), st


def check(dt, P, leaf=32):
    e, d, st = run(dt, P, leaf)
    te, td2 = oemst.canonical(*oemst.emst_kruskal(P))
    ge, gd = oemst.canonical(e, d)
    assert np.array_equal(ge, te)
    assert np.array_equal(gd, np.sqrt(td2).astype(np.float32))
    return st


def test_unit_square_ties(dt):
    P = np.array([[0, 0], [1, 0], [1, 1], [0, 1]], dtype=np.float32)
    for leaf in (1, 2, 4):
        e, _, _ = run(dt, P, leaf)
        assert oemst.canonical(e, np.zeros(3))[0].tolist() == [[0, 1], [0, 3], [1, 2]]


def test_points_on_a_line(dt):
    P = np.zeros((300, 3), dtype=np.float32)
    P[:, 0] = np.random.default_rng(1).permutation(300)
    check(dt, P, leaf=8)


@pytest.mark.parametrize("n,d,leaf", [(2, 3, 32), (3, 2, 1), (17, 5, 2), (500, 2, 8),
                                      (3000, 3, 32), (2000, 8, 16), (1500, 16, 32), (600, 33, 8),
                                      (400, 64, 4), (1000, 1, 16)])
def test_gaussian(dt, n, d, leaf):
    P = np.random.default_rng(n + d).normal(size=(n, d)).astype(np.float32)
    check(dt, P, leaf)


def test_lattice_with_duplicates(dt):
    # zero-length edges and many equal lengths: the order decides
    P = np.random.default_rng(7).integers(0, 8, size=(2500, 2)).astype(np.float32)
    check(dt, P, leaf=8)


def test_far_clusters(dt):
    g = np.random.default_rng(9)
    P = (g.normal(size=(2400, 4)) + 60 * g.integers(0, 6, size=(2400, 1))).astype(np.float32)
    st = check(dt, P, leaf=16)
    assert st["point_pairs"] > 0


def test_gmm16_sample(dt):
    W = inputs.gmm16(n_ref=4000, n_query=10)
    check(dt, W.ref)


def test_one_point_and_errors(dt):
    t = dt.dtree_build(torch.zeros((1, 3), dtype=torch.float32, device="cuda"), 8)
    try:
        e, d = dt.dtree_emst(t)
        assert e.shape == (0, 2) and d.shape == (0,)
    finally:
        t.free()
    t = dt.dtree_build(torch.from_numpy(inputs.uniform(100, 3, 2)).cuda(), 8)
    try:
        with pytest.raises(dt.DTreeError) as ex:
            dt.dtree_emst(t, precision="bf16")
        assert ex.value.status == -7
    finally:
        t.free()
