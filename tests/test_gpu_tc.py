"""Tensor-core (tcgen05) path: one-tile layout check, then kNN parity with the
oracle in BF16 and TF32 (exactness comes from the error band + float64 re-rank)."""
import os

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


def rounded(x, fmt):
    if fmt == "bf16":
        return x.to(torch.bfloat16).to(torch.float64)
    # TF32, round to nearest (ties away from zero): keep 10 explicit mantissa bits
    b = x.contiguous().view(torch.int32).to(torch.int64)
    b = (b + 0x1000) & ~0x1FFF
    return b.to(torch.int32).view(torch.float32).to(torch.float64)


@pytest.mark.parametrize("fmt", ["bf16", "tf32"])
@pytest.mark.parametrize("K", [3, 8, 16, 24, 32, 64])
def test_mma_tile_layout(dt, fmt, K):
    g = torch.Generator().manual_seed(K)
    A = torch.randn(128, K, generator=g).cuda()
    B = torch.randn(128, K, generator=g).cuda()
    out = dt.dtree_debug_mma(A, B, fmt).double()
    ref = rounded(A, fmt) @ rounded(B, fmt).T
    scale = (rounded(A, fmt).abs() @ rounded(B, fmt).abs().T)
    err = ((out - ref).abs() / (scale + 1e-30)).max().item()
    assert err < 64 * 2.0 ** -23, err


@pytest.mark.parametrize("prec", ["bf16", "tf32"])
@pytest.mark.parametrize("d", [3, 8, 16, 32, 64])
@pytest.mark.parametrize("mono", [True, False])
def test_tc_parity_dims(dt, prec, d, mono):
    R = inputs.gaussian(4001, d, 500 + d)
    Q = None if mono else inputs.uniform(1203, d, 600 + d) * 2 - 1
    for k in (1, 5, 10):
        idx, dist = run(dt, R, Q, k, 16, precision=prec)
        ti, td = truth(R, Q, k)
        compare(idx, dist, ti, td, k)


@pytest.mark.parametrize("prec", ["bf16", "tf32"])
def test_tc_gmm16_scaled(dt, prec):
    W = inputs.gmm16(n_ref=200_000, n_query=20_000)
    idx, dist, st = run(dt, W.ref, W.query, W.k, W.leaf_size, stats=True, precision=prec)
    ti, td = truth(W.ref, W.query, W.k)
    r = compare(idx, dist, ti, td, W.k)
    assert r["exact"] + r["exempt"] == 20_000
    # the band overflows for few queries (d = 16: TF32, and BF16 as hi + lo
    # pairs); those are recomputed exactly, so this bounds cost, not correctness
    assert st["fallback_queries"] <= 20


@pytest.mark.parametrize("prec", ["bf16", "tf32"])
def test_tc_duplicates(dt, prec):
    R = inputs.duplicate_heavy(3000, 16, 7)
    Q = inputs.duplicate_heavy(900, 16, 8)
    for q in (None, Q):
        idx, dist = run(dt, R, q, 10, 16, precision=prec)
        ti, td = truth(R, q, 10)
        compare(idx, dist, ti, td, 10)


@pytest.mark.parametrize("prec", ["bf16", "tf32"])
def test_tc_offset_cloud(dt, prec):
    # a cloud far from the origin: centring on the reference root box keeps
    # the rounded coordinates small
    R = inputs.gaussian(20000, 16, 31) + 1000.0
    Q = inputs.gaussian(3000, 16, 32) + 1000.0
    idx, dist = run(dt, R.astype(np.float32), Q.astype(np.float32), 10, 32, precision=prec)
    ti, td = truth(R.astype(np.float32), Q.astype(np.float32), 10)
    compare(idx, dist, ti, td, 10)


@pytest.mark.parametrize("prec", ["bf16", "tf32"])
def test_tc_k_values(dt, prec):
    R = inputs.gaussian(6000, 32, 41)
    Q = inputs.gaussian(1500, 32, 42)
    for k in (1, 2, 7, 15, 31, 34, 47, 50, 63):
        idx, dist = run(dt, R, Q, k, 32, precision=prec)
        ti, td = truth(R, Q, k)
        compare(idx, dist, ti, td, k)


@pytest.mark.skipif(os.environ.get("DTREE_SKIP_FULL") == "1", reason="full-size run disabled")
def test_tc_gmm16_full_size_sampled(dt):
    W = inputs.gmm16()
    idx, dist = run(dt, W.ref, W.query, W.k, W.leaf_size, precision="bf16")
    rng = np.random.default_rng(6)
    sample = np.sort(rng.choice(len(W.query), 256, replace=False))
    ti, td = truth(W.ref, W.query, W.k, sample)
    r = compare(idx[sample], dist[sample], ti, td, W.k)
    assert r["exact"] + r["exempt"] == 256


@pytest.mark.parametrize("prec", ["bf16", "tf32"])
@pytest.mark.parametrize("d", [5, 16, 64])
@pytest.mark.parametrize("leaf", [1, 5, 20, 37, 300])
def test_tc_leaf_sizes(dt, prec, d, leaf):
    # leaves of every size pad to whole 8-row groups of the operand rows; a
    # leaf wider than a tile (300 > 256 or 128 points) is split across tiles
    R = inputs.gaussian(7001, d, 700 + d + leaf)
    Q = inputs.gaussian(1501, d, 800 + d + leaf)
    for q, k in ((Q, 10), (None, 3)):
        idx, dist = run(dt, R, q, k, leaf, precision=prec)
        ti, td = truth(R, q, k)
        compare(idx, dist, ti, td, k)


@pytest.mark.parametrize("prec", ["bf16", "tf32"])
def test_tc_powerlaw64_k50(dt, prec):
    """The combined workload's shape (d = 64, k = 50) at 60k x 6k: every query."""
    W = inputs.powerlaw64(n_ref=60_000, n_query=6_000)
    assert W.k == 50
    idx, dist, st = run(dt, W.ref, W.query, W.k, W.leaf_size, stats=True, precision=prec)
    ti, td = truth(W.ref, W.query, W.k)
    r = compare(idx, dist, ti, td, W.k)
    assert r["exact"] + r["exempt"] == 6_000
    # lists of 64 hold the band: overflows are rare (they are recomputed
    # exactly, so this bounds cost, not correctness)
    assert st["fallback_queries"] <= 60, st["fallback_queries"]
    # monochromatic, with the self-match excluded
    idx, dist = run(dt, W.ref[:20_000], None, W.k, W.leaf_size, precision=prec)
    ti, td = truth(W.ref[:20_000], None, W.k)
    compare(idx, dist, ti, td, W.k)


@pytest.mark.skipif(os.environ.get("DTREE_SKIP_FULL") == "1", reason="full-size run disabled")
def test_tc_powerlaw64_full_size_sampled(dt):
    """2M x 2M, d = 64, k = 50 in split BF16: 256 sampled queries against brute
    force, and fewer than 0.1% of the queries recomputed."""
    W = inputs.powerlaw64()
    idx, dist, st = run(dt, W.ref, W.query, W.k, W.leaf_size, stats=True, precision="bf16")
    rng = np.random.default_rng(7)
    sample = np.sort(rng.choice(len(W.query), 256, replace=False))
    ti, td = truth(W.ref, W.query, W.k, sample)
    r = compare(idx[sample], dist[sample], ti, td, W.k)
    assert r["exact"] + r["exempt"] == 256
    assert st["fallback_queries"] < len(W.query) // 1000, st["fallback_queries"]


@pytest.mark.parametrize("fmt", ["bf16", "tf32"])
@pytest.mark.parametrize("K", [8, 16, 64])
@pytest.mark.parametrize("shift", [0.0, -3.0])
def test_tmem_load_reduced_minimum(dt, fmt, K, shift):
    """The epilogue skips 64 columns on the minimum that tcgen05.ld.red
    returns with the load: on one accumulator tile (negative and positive
    values, with shift), the 32- and 64-column minima the loads reduce to
    equal the float32 minima of the columns read back."""
    g = torch.Generator().manual_seed(100 + K)
    A = torch.randn(128, K, generator=g).cuda()
    B = (torch.randn(128, K, generator=g) + shift).cuda()
    out, m32, m64 = dt.dtree_debug_tmem_min(A, B, fmt)
    assert torch.equal(m32, out.view(128, 4, 32).amin(dim=2))
    assert torch.equal(m64, out.view(128, 2, 64).amin(dim=2))
