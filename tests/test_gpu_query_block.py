"""Query blocks of more than 128 queries: the traversal's unit is a larger
query-tree node, processed as chunks of 128 that share its candidate leaves.
The lists must equal the FP64 oracle's whatever the block size."""
import ctypes

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


@pytest.mark.parametrize("qb", [200, 256, 512])
@pytest.mark.parametrize("prec", ["fp32", "bf16"])
@pytest.mark.parametrize("d", [3, 16, 64])
@pytest.mark.parametrize("mono", [True, False])
def test_large_query_blocks_match_the_oracle(dt, qb, prec, d, mono):
    R = inputs.gaussian(12_001, d, 8100 + d)
    Q = None if mono else inputs.uniform(3_003, d, 8200 + d) * 2 - 1
    for k in (1, 10):
        idx, dist = run(dt, R, Q, k, 16, precision=prec, query_block=qb)
        ti, td = truth(R, Q, k)
        compare(idx, dist, ti, td, k)


def test_large_blocks_give_the_same_lists_as_small_ones(dt):
    W = inputs.powerlaw64(n_ref=60_000, n_query=6_000)
    i0, d0 = run(dt, W.ref, W.query, W.k, W.leaf_size, precision="bf16", query_block=128)
    for qb in (256, 512):
        i1, d1, st = run(dt, W.ref, W.query, W.k, W.leaf_size, precision="bf16", query_block=qb, stats=True)
        assert np.array_equal(i0, i1) and np.array_equal(d0, d1), qb
        # blocks of up to qb queries: fewer blocks than with 128
        assert st["query_blocks"] <= (6_000 + 127) // 128


def test_batch_with_large_per_problem_blocks(dt):
    probs, trees = [], []
    for i, (n, d, qb) in enumerate([(9_000, 8, 512), (5_000, 32, 256), (7_000, 3, 0)]):
        X = inputs.gaussian(n, d, 8300 + i)
        tr = dt.dtree_build(torch.from_numpy(X).cuda(), 16)
        trees.append((tr, X))
        probs.append((None, tr, 5, qb))
    try:
        outs = dt.dtree_knn_batch(probs, precision="bf16")
        for (tr, X), (idx, dist) in zip(trees, outs):
            ti, td = truth(X, None, 5)
            compare(idx.cpu().numpy(), dist.cpu().numpy(), ti, td, 5)
    finally:
        for tr, _ in trees:
            tr.free()


def test_query_block_beyond_512_is_rejected(dt):
    R = torch.from_numpy(inputs.uniform(2000, 3, 8400)).cuda()
    tr = dt.dtree_build(R, 16)
    try:
        with pytest.raises(dt.DTreeError) as e:
            dt.dtree_knn(None, tr, 3, query_block=513)
        assert e.value.status == -1  # DTREE_ERR_INVALID_ARG
    finally:
        tr.free()
