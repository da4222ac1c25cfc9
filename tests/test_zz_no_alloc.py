"""dtree_knn_noalloc: the search with its scratch in a fixed static device
array.  Two calls in a row must each give exactly dtree_knn's result, and
neither may allocate device memory.  Self-contained, so it passes alone and
after the rest of the suite."""
import numpy as np
import pytest
import torch

from paper_1304_4327_gb300 import inputs

pytestmark = pytest.mark.gpu

DTREE_ERR_INVALID_ARG = -1
DTREE_ERR_TOO_LARGE = -8


@pytest.fixture(scope="module")
def dt():
    from paper_1304_4327_gb300 import build
    build.build()
    from paper_1304_4327_gb300 import dtree
    return dtree


def _pair(dt, R, Q, k, leaf, prec):
    tr = dt.dtree_build(torch.from_numpy(R).cuda(), leaf)
    tq = None if Q is None else dt.dtree_build(torch.from_numpy(Q).cuda(), leaf)
    try:
        i0, d0 = dt.dtree_knn(tq, tr, k, precision=prec)
        nq = tr.n if tq is None else tq.n
        oi = torch.empty((nq, k), dtype=torch.int64, device="cuda")
        od = torch.empty((nq, k), dtype=torch.float32, device="cuda")
        torch.cuda.synchronize()
        a0 = dt.alloc_count()
        for _ in range(2):
            oi.fill_(-7)
            od.fill_(float("nan"))
            dt.dtree_knn_noalloc(tq, tr, k, oi, od, precision=prec)
            torch.cuda.synchronize()
            assert torch.equal(oi, i0)
            assert torch.equal(od, d0)
        assert dt.alloc_count() == a0, "the no-allocation entry point allocated"
    finally:
        tr.free()
        if tq is not None:
            tq.free()


@pytest.mark.parametrize("prec", ["fp32", "bf16"])
def test_two_calls_match_dtree_knn_bichromatic(dt, prec):
    R = inputs.gaussian(60_000, 16, 4101)
    Q = inputs.gaussian(20_000, 16, 4102)
    _pair(dt, R, Q, 10, 32, prec)


def test_two_calls_match_dtree_knn_monochromatic(dt):
    X = inputs.uniform(30_000, 3, 4103)
    _pair(dt, X, None, 5, 20, "fp32")


def test_duplicates_use_the_fallback_in_the_fixed_scratch(dt):
    R = inputs.duplicate_heavy(4000, 3, 4104)
    Q = inputs.duplicate_heavy(1500, 3, 4105)
    _pair(dt, R, Q, 10, 16, "fp32")


def test_largest_query_count(dt):
    R = inputs.uniform(100_000, 8, 4106)
    Q = inputs.uniform(dt.NOALLOC_MAX_QUERIES, 8, 4107)
    _pair(dt, R, Q, 4, 32, "fp32")


def test_rejects_sizes_beyond_the_maximum(dt):
    R = torch.from_numpy(inputs.uniform(2000, 3, 4108)).cuda()
    Q = torch.from_numpy(inputs.uniform(dt.NOALLOC_MAX_QUERIES + 1, 3, 4109)).cuda()
    tr = dt.dtree_build(R, 16)
    tq = dt.dtree_build(Q, 16)
    try:
        oi = torch.empty((tq.n, 3), dtype=torch.int64, device="cuda")
        od = torch.empty((tq.n, 3), dtype=torch.float32, device="cuda")
        a0 = dt.alloc_count()
        with pytest.raises(dt.DTreeError) as e:
            dt.dtree_knn_noalloc(tq, tr, 3, oi, od)
        assert e.value.status == DTREE_ERR_TOO_LARGE
        assert dt.alloc_count() == a0
    finally:
        tr.free()
        tq.free()


def test_candidate_pairs_beyond_the_array_are_refused(dt):
    # d = 64 power-law points: nearly every (query block, leaf) pair survives
    # the bound, so 20k queries against 400k references in leaves of 4 points
    # need far more candidate-pair storage than the array holds; the device
    # reports it and the call returns DTREE_ERR_TOO_LARGE without allocating
    W = inputs.powerlaw64(n_ref=400_000, n_query=20_000)
    tr = dt.dtree_build(torch.from_numpy(W.ref).cuda(), 4)
    tq = dt.dtree_build(torch.from_numpy(W.query).cuda(), 4)
    try:
        oi = torch.empty((tq.n, 5), dtype=torch.int64, device="cuda")
        od = torch.empty((tq.n, 5), dtype=torch.float32, device="cuda")
        torch.cuda.synchronize()
        a0 = dt.alloc_count()
        with pytest.raises(dt.DTreeError) as e:
            dt.dtree_knn_noalloc(tq, tr, 5, oi, od)
        assert e.value.status == DTREE_ERR_TOO_LARGE
        assert dt.alloc_count() == a0
    finally:
        tr.free()
        tq.free()
    # a problem that fits still gives dtree_knn's result afterwards
    _pair(dt, W.ref[:50_000], W.query[:5_000], 5, 32, "fp32")
