"""Parity of the CUDA kNN path (through the C ABI) with the CPU oracle."""
import os

import numpy as np
import pytest
import torch

import oracle
from paper_1304_4327_gb300 import inputs
from parity import compare

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def dt():
    from paper_1304_4327_gb300 import build
    build.build()
    from paper_1304_4327_gb300 import dtree
    return dtree


def run(dt, ref, query, k, leaf=32, stats=False, **kw):
    r = torch.from_numpy(np.ascontiguousarray(ref)).cuda()
    q = None if query is None else torch.from_numpy(np.ascontiguousarray(query)).cuda()
    tr = dt.dtree_build(r, leaf)
    tq = None if q is None else dt.dtree_build(q, leaf)
    try:
        out = dt.dtree_knn(tq, tr, k, with_stats=stats, **kw)
    finally:
        tr.free()
        if tq is not None:
            tq.free()
    res = (out[0].cpu().numpy(), out[1].cpu().numpy())
    return res + ((out[2],) if stats else ())


def truth(ref, query, k, sample=None):
    m = ref.shape[0]
    kk = k + 1 if k + 1 <= (m - 1 if query is None else m) else k
    if sample is None:
        return oracle.knn_brute(ref, query, kk)
    if query is None:
        return oracle.knn_brute(ref, ref[sample], kk, self_idx=np.asarray(sample, dtype=np.int64))
    return oracle.knn_brute(ref, query[sample], kk)


def check(dt, ref, query, k, leaf=32, **kw):
    idx, dist = run(dt, ref, query, k, leaf, **kw)
    ti, td = truth(ref, query, k)
    return compare(idx, dist, ti, td, k)


# ---------------------------------------------------------------------------
# the paper's worked example and the first workload
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("k", [1, 2, 3, 4])
@pytest.mark.parametrize("leaf", [1, 2, 5])
def test_figure1(dt, k, leaf):
    from test_oracle import load_figure1
    P, I, D = load_figure1()
    idx, dist = run(dt, P, None, k, leaf)
    assert np.array_equal(idx, I[:, :k])
    assert np.array_equal(dist, np.sqrt(D[:, :k]).astype(np.float32))


def test_mono_uniform_10k(dt):
    W = inputs.mono_uniform()
    idx, dist, st = run(dt, W.ref, None, W.k, W.leaf_size, stats=True)
    ti, td = truth(W.ref, None, W.k)
    r = compare(idx, dist, ti, td, W.k)
    assert r["exact"] == len(W.ref)
    n = len(W.ref)
    assert 0 < st["point_pairs"] < n * n // 4          # the bound prunes
    assert st["node_pairs_pruned"] > 0
    assert st["kernel_launches"] > 0


# ---------------------------------------------------------------------------
# sweeps over dimension, k, distribution, mono / bichromatic
# ---------------------------------------------------------------------------

GEN = {
    "uniform": inputs.uniform,
    "gaussian": inputs.gaussian,
    "collinear": inputs.collinear,
}


@pytest.mark.parametrize("d", [1, 2, 3, 5, 8, 12, 16, 32, 64])
@pytest.mark.parametrize("mono", [True, False])
def test_sweep_dims(dt, d, mono):
    for kind, gen in GEN.items():
        R = gen(3001, d, 10 * d + 1)
        Q = None if mono else gen(1203, d, 10 * d + 2)
        for k in (1, 5, 10):
            check(dt, R, Q, k, leaf=16)


@pytest.mark.parametrize("k", [1, 3, 7, 8, 15, 16, 31])
def test_sweep_k(dt, k):
    R = inputs.gaussian(5000, 6, 77)
    Q = inputs.uniform(777, 6, 78)
    check(dt, R, Q, k, leaf=20)
    check(dt, R, None, k, leaf=20)


@pytest.mark.parametrize("leaf", [1, 2, 3, 7, 64, 300, 1024])
def test_leaf_sizes(dt, leaf):
    R = inputs.uniform(6000, 3, 91)
    Q = inputs.uniform(2500, 3, 92)
    check(dt, R, Q, 5, leaf=leaf)
    check(dt, R, None, 5, leaf=leaf)


@pytest.mark.parametrize("qb", [16, 32, 64, 128])
def test_query_block(dt, qb):
    R = inputs.gaussian(8000, 8, 93)
    Q = inputs.gaussian(3000, 8, 94)
    check(dt, R, Q, 10, leaf=32, query_block=qb)


def test_duplicates_take_the_float64_path(dt):
    R = inputs.duplicate_heavy(4000, 3, 5)
    Q = inputs.duplicate_heavy(1500, 3, 6)
    idx, dist, st = run(dt, R, Q, 10, 16, stats=True)
    ti, td = truth(R, Q, 10)
    compare(idx, dist, ti, td, 10)
    # 7 distinct points: every k-th distance is an exact tie shared by many
    # points, so the float32 band overflows as well and float64 decides
    assert st["fallback_queries"] > 0 and st["fallback64_queries"] > 0
    idx, dist, st = run(dt, R, None, 10, 16, stats=True)
    ti, td = truth(R, None, 10)
    compare(idx, dist, ti, td, 10)


def test_lattice_ties(dt):
    X = inputs.lattice([20, 20, 5])
    idx, dist = run(dt, X, None, 6, 8)
    ti, td = truth(X, None, 6)
    compare(idx, dist, ti, td, 6)


# ---------------------------------------------------------------------------
# edge cases of the problem statement
# ---------------------------------------------------------------------------

def test_tiny_inputs(dt):
    X = np.array([[0.0, 0.0], [1.0, 0.0]], dtype=np.float32)
    idx, dist = run(dt, X, None, 1, 2)
    assert idx.tolist() == [[1], [0]] and dist.tolist() == [[1.0], [1.0]]
    R = inputs.uniform(3, 4, 1)
    Q = inputs.uniform(1, 4, 2)
    check(dt, R, Q, 2, leaf=2)


def test_k_max(dt):
    R = inputs.uniform(30, 3, 3)
    Q = inputs.uniform(17, 3, 4)
    check(dt, R, None, 29, leaf=4)                     # k = m - 1, monochromatic
    check(dt, R, Q, 29, leaf=4)                        # k = m - 1 < m, bichromatic


def test_invalid_k(dt):
    R = torch.from_numpy(inputs.uniform(50, 3, 5)).cuda()
    tr = dt.dtree_build(R, 8)
    try:
        for k in (0, -1, 50):
            with pytest.raises(dt.DTreeError) as e:
                dt.dtree_knn(None, tr, k)
            assert e.value.status == -2
        tq = dt.dtree_build(R[:10].contiguous(), 8)
        with pytest.raises(dt.DTreeError):
            dt.dtree_knn(tq, tr, 51)
        tq.free()
    finally:
        tr.free()


def test_deterministic(dt):
    R = inputs.gaussian(20000, 16, 9)
    Q = inputs.gaussian(5000, 16, 10)
    a = run(dt, R, Q, 10)
    b = run(dt, R, Q, 10)
    assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1])


# ---------------------------------------------------------------------------
# the tree itself
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("n,d,leaf", [(10000, 3, 20), (70001, 16, 32), (5000, 64, 8), (3000, 8, 500)])
def test_tree_invariants(dt, n, d, leaf):
    X = inputs.gaussian(n, d, n + d)
    tr = dt.dtree_build(torch.from_numpy(X).cuda(), leaf)
    try:
        ex = {k: v.cpu().numpy() for k, v in dt.dtree_export(tr).items()}
        depth, leaves = tr.depth, tr.leaves
    finally:
        tr.free()
    perm, box, lam, beg, cnt = ex["perm"], ex["box"], ex["lambda"], ex["begin"], ex["count"]
    assert np.array_equal(np.sort(perm), np.arange(n))
    nodes = 2 * leaves - 1
    assert leaves == 2 ** depth and box.shape == (nodes, 2, d)
    leaf_cnt = cnt[leaves - 1:]
    assert leaf_cnt.max() <= max(leaf, 2) and leaf_cnt.min() >= 1
    P = X[perm].astype(np.float64)
    for i in range(nodes):
        pts = P[beg[i]:beg[i] + cnt[i]]
        assert np.all(pts.min(0) == box[i, 0]) and np.all(pts.max(0) == box[i, 1]), i
        centre = 0.5 * (box[i, 0].astype(np.float32) + box[i, 1].astype(np.float32))
        exact = np.sqrt(((pts - centre.astype(np.float64)) ** 2).sum(1)).max()
        assert lam[i] >= exact, (i, lam[i], exact)
        if i > 0:
            p = (i - 1) // 2
            assert np.all(box[i, 0] >= box[p, 0]) and np.all(box[i, 1] <= box[p, 1])
        if i < leaves - 1:
            l, r = 2 * i + 1, 2 * i + 2
            assert cnt[l] == cnt[i] // 2 and cnt[l] + cnt[r] == cnt[i]
            assert beg[l] == beg[i] and beg[r] == beg[i] + cnt[l]


# ---------------------------------------------------------------------------
# the workloads at larger scale
# ---------------------------------------------------------------------------

def test_gmm16_scaled(dt):
    W = inputs.gmm16(n_ref=200_000, n_query=20_000)
    r = check(dt, W.ref, W.query, W.k, W.leaf_size)
    assert r["exact"] + r["exempt"] == 20_000


def test_latent3_scaled(dt):
    W = inputs.latent3(n_ref=300_000, n_query=20_000, n_train=10)
    check(dt, W.ref, W.query, W.k, W.leaf_size)


def test_powerlaw64_scaled(dt):
    W = inputs.powerlaw64(n_ref=60_000, n_query=6_000)
    check(dt, W.ref, W.query, 31, W.leaf_size)


def test_powerlaw64_k50_scaled(dt):
    # the power-law workload's own k (lists of 64), on the CUDA cores and the
    # tensor cores
    W = inputs.powerlaw64(n_ref=40_000, n_query=3_000)
    assert W.k == 50
    check(dt, W.ref, W.query, W.k, W.leaf_size)
    check(dt, W.ref[:20_000], None, W.k, W.leaf_size)
    for prec in ("bf16", "tf32"):
        check(dt, W.ref, W.query, W.k, W.leaf_size, precision=prec)


@pytest.mark.parametrize("prec", ["fp32", "tf32", "bf16"])
def test_k_above_63_is_unsupported(dt, prec):
    R = inputs.gaussian(3000, 8, 11)
    with pytest.raises(dt.DTreeError) as e:
        run(dt, R, None, 64, 16, precision=prec)
    assert e.value.status == -7          # DTREE_ERR_UNSUPPORTED


@pytest.mark.parametrize("k", [32, 47, 48, 63])
def test_large_k(dt, k):
    R = inputs.gaussian(6000, 5, 200 + k)
    Q = inputs.uniform(900, 5, 300 + k)
    check(dt, R, Q, k, leaf=16)
    check(dt, R, None, k, leaf=16)
    with pytest.raises(dt.DTreeError) as e:
        run(dt, R, Q, 64, 16)
    assert e.value.status == -7


def test_batched_problems_scaled(dt):
    for spec in inputs.batched_specs()[:24]:
        W = inputs.batched_problem(spec, n_cap=20_000)
        check(dt, W.ref, None, W.k, 16)


@pytest.mark.skipif(os.environ.get("DTREE_SKIP_FULL") == "1", reason="full-size run disabled")
def test_gmm16_full_size_sampled(dt):
    """4M references x 1M queries, d=16, k=10: 256 sampled queries vs brute force."""
    W = inputs.gmm16()
    idx, dist = run(dt, W.ref, W.query, W.k, W.leaf_size)
    rng = np.random.default_rng(5)
    sample = np.sort(rng.choice(len(W.query), 256, replace=False))
    ti, td = truth(W.ref, W.query, W.k, sample)
    r = compare(idx[sample], dist[sample], ti, td, W.k)
    assert r["exact"] + r["exempt"] == 256
