"""dtree_knn_batch: many problems in one call give exactly the results of one
dtree_knn call per problem, and those of the oracle."""
import numpy as np
import pytest
import torch

from paper_1304_4327_gb300 import inputs
from parity import compare
from test_gpu_knn import truth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def dt():
    from paper_1304_4327_gb300 import build
    build.build()
    from paper_1304_4327_gb300 import dtree
    return dtree


def _trees(dt, probs, leaf):
    out = []
    for R, Q, k in probs:
        tr = dt.dtree_build(torch.from_numpy(np.ascontiguousarray(R)).cuda(), leaf)
        tq = None if Q is None else dt.dtree_build(torch.from_numpy(np.ascontiguousarray(Q)).cuda(), leaf)
        out.append((tq, tr, k))
    return out


def _free(trees):
    for tq, tr, _ in trees:
        tr.free()
        if tq is not None:
            tq.free()


def _check(dt, probs, leaf=16, precision="fp32", **kw):
    trees = _trees(dt, probs, leaf)
    try:
        outs, st = dt.dtree_knn_batch(trees, precision=precision, with_stats=True, **kw)
        for (tq, tr, k), (R, Q, _), (oi, od) in zip(trees, probs, outs):
            si, sd = dt.dtree_knn(tq, tr, k, precision=precision, **kw)
            assert torch.equal(oi, si) and torch.equal(od, sd)
            ti, td = truth(R, Q, k)
            compare(oi.cpu().numpy(), od.cpu().numpy(), ti, td, k)
        return st
    finally:
        _free(trees)


def test_batched_workload_problems(dt):
    # the batched workload's shapes (d in {3, 8, 32}, k in {1, 10}), capped in size
    specs = inputs.batched_specs()[:40]
    probs = []
    for spec in specs:
        W = inputs.batched_problem(spec, n_cap=12_000)
        probs.append((W.ref, None, W.k))
    st = _check(dt, probs)
    assert st["query_blocks"] > 0 and st["point_pairs"] > 0


def test_mixed_problems_one_group(dt):
    # one width bucket: mono and bichromatic, different k, tiny and larger
    probs = [
        (inputs.gaussian(5000, 6, 1), inputs.uniform(700, 6, 2), 10),
        (inputs.uniform(3000, 5, 3), None, 1),
        (np.array([[0.0] * 7, [1.0] + [0.0] * 6], dtype=np.float32), None, 1),
        (inputs.uniform(4, 8, 4), inputs.uniform(3, 8, 5), 3),
        (inputs.duplicate_heavy(2500, 7, 6), None, 12),
        (inputs.gaussian(20000, 8, 7), inputs.gaussian(4000, 8, 8), 31),
    ]
    _check(dt, probs)


@pytest.mark.parametrize("prec", ["tf32", "bf16"])
def test_tensor_core_batch(dt, prec):
    probs = [
        (inputs.gaussian(30000, 16, 11), inputs.gaussian(3000, 16, 12), 10),
        (inputs.uniform(8000, 13, 13), None, 5),
        (inputs.gaussian(6000, 32, 14), inputs.uniform(900, 32, 15), 7),
        (inputs.gaussian(2000, 16, 16), None, 1),
    ]
    _check(dt, probs, leaf=32, precision=prec)


def test_per_problem_query_block(dt):
    R = inputs.gaussian(9000, 8, 21)
    Q = inputs.gaussian(2500, 8, 22)
    trees = _trees(dt, [(R, Q, 6), (R, None, 4)], 16)
    try:
        (tq, tr, _), (_, tr2, _) = trees
        outs = dt.dtree_knn_batch([(tq, tr, 6, 32), (None, tr2, 4, 128)])
        a = dt.dtree_knn(tq, tr, 6, query_block=32)
        b = dt.dtree_knn(None, tr2, 4, query_block=128)
        assert torch.equal(outs[0][0], a[0]) and torch.equal(outs[1][0], b[0])
        assert torch.equal(outs[0][1], a[1]) and torch.equal(outs[1][1], b[1])
    finally:
        _free(trees)


def test_empty_and_invalid_batches(dt):
    assert dt.dtree_knn_batch([]) == []
    R = torch.from_numpy(inputs.uniform(100, 3, 31)).cuda()
    tr = dt.dtree_build(R, 8)
    try:
        with pytest.raises(dt.DTreeError) as e:
            dt.dtree_knn_batch([(None, tr, 5), (None, tr, 100)])
        assert e.value.status == -2
        with pytest.raises(dt.DTreeError) as e:
            dt.dtree_knn_batch([(None, tr, 5, 8)])
        assert e.value.status == -1
    finally:
        tr.free()


def test_autotuned_batch(dt, tmp_path):
    from paper_1304_4327_gb300 import autotune
    specs = inputs.batched_specs()[:12]
    probs, host = [], []
    for spec in specs:
        W = inputs.batched_problem(spec, n_cap=8_000)
        probs.append((torch.from_numpy(W.ref).cuda(), None, W.k))
        host.append((W.ref, W.k))
    tuner = autotune.Autotuner(str(tmp_path / "tune.json"), repeats=1)
    outs = autotune.run_batch(probs, tuner=tuner)
    for (R, k), (oi, od) in zip(host, outs):
        ti, td = truth(R, None, k)
        compare(oi.cpu().numpy(), od.cpu().numpy(), ti, td, k)
    assert tuner.table and all(v[0] in autotune.LEAVES and v[1] in autotune.BLOCKS
                               for v in tuner.table.values())
    # a second run answers every class from the cache
    again = autotune.Autotuner(str(tmp_path / "tune.json"))
    assert again.table == tuner.table
    n_timed = len(tuner.timings)
    autotune.run_batch(probs, tuner=tuner)
    assert len(tuner.timings) == n_timed
