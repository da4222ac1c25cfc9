"""The learned leaf proposal: the network's kernels against the FP64 oracle,
training on the method's own answers, and exact search with the proposal
(which only reorders work) together with what it gains."""
import numpy as np
import pytest
import torch

from oracle import mlp as omlp
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


def _rel(a, b):
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-30))


@pytest.mark.parametrize("n,d,C", [(96, 8, 512), (130, 3, 200), (256, 16, 1024), (37, 33, 129)])
def test_loss_and_gradients_match_the_oracle(dt, n, d, C):
    p = omlp.init(d, C, seed=n + d + C, scale=0.7)
    g = np.random.default_rng(C)
    X = g.normal(size=(n, d))
    T = g.random(size=(n, C)) * (g.random(size=(n, C)) < 0.05)
    T[:, 0] += 1e-3
    T /= T.sum(axis=1, keepdims=True)
    L, G = omlp.loss_grad(p, X, T)
    params = [torch.from_numpy(p[k].astype(np.float32)).cuda() for k in omlp.NAMES]
    Lg, grads = dt.dtree_mlp_loss_grad(params, torch.from_numpy(X.astype(np.float32)).cuda(),
                                       torch.from_numpy(T.astype(np.float32)).cuda())
    # FP16 operands (unit roundoff 2^-11) with FP32 accumulation
    assert Lg == pytest.approx(L, rel=5e-3)
    for name, gg in zip(omlp.NAMES, grads):
        err = _rel(gg.cpu().numpy().astype(np.float64), G[name])
        assert err < 3e-2, (name, err)


def _setup(dt, n_ref, n_query, n_train, leaf=32):
    W = inputs.latent3(n_ref=n_ref, n_query=n_query, n_train=n_train)
    tr = dt.dtree_build(torch.from_numpy(W.ref).cuda(), leaf)
    tq = dt.dtree_build(torch.from_numpy(W.query).cuda(), leaf)
    tt = dt.dtree_build(torch.from_numpy(W.extra["train"]).cuda(), leaf)
    return W, tr, tq, tt


def test_training_learns_and_search_stays_exact(dt):
    W, tr, tq, tt = _setup(dt, 200_000, 20_000, 20_000)
    try:
        model = dt.dtree_proposal_train(tr, tt, W.k, epochs=30, batch=128)
        assert model.classes >= 2
        losses = model.losses
        assert np.all(np.isfinite(losses))
        assert losses[-1] < 0.8 * losses[0], losses
        dt.dtree_attach_proposal(tr, model)
        ti, td = truth(W.ref, W.query, W.k)
        base = dt.dtree_knn(tq, tr, W.k, with_stats=True)
        for M in (1, 4, 8):
            idx, dist, st = dt.dtree_knn(tq, tr, W.k, with_stats=True, proposal=M)
            compare(idx.cpu().numpy(), dist.cpu().numpy(), ti, td, W.k)
            assert torch.equal(idx, base[0]) and torch.equal(dist, base[1])
        # the gain: a tighter B before the traversal leaves fewer candidate
        # leaf pairs for the BaseCase pass
        _, _, st4 = dt.dtree_knn(tq, tr, W.k, with_stats=True, proposal=4)
        print("without proposal:", {k: base[2][k] for k in ("leaf_pairs_emitted", "point_pairs",
                                                             "seed_point_pairs")})
        print("with proposal (M=4):", {k: st4[k] for k in ("leaf_pairs_emitted", "point_pairs",
                                                          "seed_point_pairs")})
        assert st4["leaf_pairs_emitted"] < base[2]["leaf_pairs_emitted"]
        # bichromatic and monochromatic batches with the proposal
        outs = dt.dtree_knn_batch([(tq, tr, W.k), (None, tr, 3)], proposal=4)
        assert torch.equal(outs[0][0], base[0])
        mi, md = dt.dtree_knn(None, tr, 3)
        assert torch.equal(outs[1][0], mi) and torch.equal(outs[1][1], md)
        dt.dtree_attach_proposal(tr, None)
        model.free()
    finally:
        for t in (tr, tq, tt):
            t.free()


def test_proposal_needs_a_model(dt):
    R = torch.from_numpy(inputs.uniform(5000, 4, 3)).cuda()
    tr = dt.dtree_build(R, 16)
    try:
        with pytest.raises(dt.DTreeError) as e:
            dt.dtree_knn(None, tr, 3, proposal=2)
        assert e.value.status == -6
        with pytest.raises(dt.DTreeError) as e:
            dt.dtree_knn(None, tr, 3, proposal=9)
        assert e.value.status == -1
    finally:
        tr.free()


def test_model_save_load_round_trip(dt, tmp_path):
    W, tr, tq, tt = _setup(dt, 100_000, 10_000, 10_000)
    tr2 = dt.dtree_build(torch.from_numpy(W.ref).cuda(), 32)
    other = dt.dtree_build(torch.from_numpy(W.ref[::2].copy()).cuda(), 32)
    try:
        model = dt.dtree_proposal_train(tr, tt, W.k, epochs=5, batch=128)
        path = tmp_path / "proposal.bin"
        dt.dtree_model_save(model, str(path))
        # a tree rebuilt from the same points accepts the file
        loaded = dt.dtree_model_load(str(path), tr2)
        assert loaded.classes == model.classes
        # the loaded weights are the saved ones: saving them again gives the same bytes
        again = tmp_path / "again.bin"
        dt.dtree_model_save(loaded, str(again))
        assert again.read_bytes() == path.read_bytes()
        # and its searches propose the same cells: identical lists and work
        dt.dtree_attach_proposal(tr, model)
        dt.dtree_attach_proposal(tr2, loaded)
        a = dt.dtree_knn(tq, tr, W.k, with_stats=True, proposal=4)
        b = dt.dtree_knn(tq, tr2, W.k, with_stats=True, proposal=4)
        assert torch.equal(a[0], b[0]) and torch.equal(a[1], b[1])
        for key in ("seed_point_pairs", "leaf_pairs_emitted", "point_pairs"):
            assert a[2][key] == b[2][key], key
        ti, td = truth(W.ref, W.query, W.k)
        compare(b[0].cpu().numpy(), b[1].cpu().numpy(), ti, td, W.k)
        # a tree of other points rejects it; a damaged file is refused
        with pytest.raises(dt.DTreeError) as e:
            dt.dtree_model_load(str(path), other)
        assert e.value.status == -1
        raw = bytearray(path.read_bytes())
        raw[100] ^= 0x40
        bad = tmp_path / "bad.bin"
        bad.write_bytes(bytes(raw))
        with pytest.raises(dt.DTreeError) as e:
            dt.dtree_model_load(str(bad), tr2)
        assert e.value.status == -9
        dt.dtree_attach_proposal(tr, None)
        dt.dtree_attach_proposal(tr2, None)
        loaded.free()
        model.free()
    finally:
        for t in (tr, tq, tt, tr2, other):
            t.free()


@pytest.mark.parametrize("prec", ["bf16", "tf32"])
def test_proposal_with_tensor_cores_is_exact(dt, prec):
    # the tensor-core search evaluates the proposed cells first in its main
    # pass; the lists, and so the results, are those of the search without it
    W, tr, tq, tt = _setup(dt, 200_000, 20_000, 20_000)
    try:
        model = dt.dtree_proposal_train(tr, tt, W.k, epochs=5, batch=128)
        dt.dtree_attach_proposal(tr, model)
        base = dt.dtree_knn(tq, tr, W.k, precision=prec)
        ti, td = truth(W.ref, W.query, W.k)
        compare(base[0].cpu().numpy(), base[1].cpu().numpy(), ti, td, W.k)
        for M in (1, 4, 8):
            idx, dist, st = dt.dtree_knn(tq, tr, W.k, precision=prec, proposal=M, with_stats=True)
            assert torch.equal(idx, base[0]) and torch.equal(dist, base[1]), M
        dt.dtree_attach_proposal(tr, None)
        model.free()
    finally:
        for t in (tr, tq, tt):
            t.free()


def test_proposal_with_tensor_cores_at_k50_d64(dt):
    W = inputs.powerlaw64(n_ref=60_000, n_query=6_000, n_train=6_000)
    tr = dt.dtree_build(torch.from_numpy(W.ref).cuda(), 32)
    tq = dt.dtree_build(torch.from_numpy(W.query).cuda(), 32)
    tt = dt.dtree_build(torch.from_numpy(W.extra["train"]).cuda(), 32)
    try:
        model = dt.dtree_proposal_train(tr, tt, W.k, epochs=5, batch=64, seed_points=256)
        dt.dtree_attach_proposal(tr, model)
        base = dt.dtree_knn(tq, tr, W.k, precision="bf16")
        idx, dist = dt.dtree_knn(tq, tr, W.k, precision="bf16", proposal=4)
        assert torch.equal(idx, base[0]) and torch.equal(dist, base[1])
        ti, td = truth(W.ref, W.query, W.k)
        compare(idx.cpu().numpy(), dist.cpu().numpy(), ti, td, W.k)
        dt.dtree_attach_proposal(tr, None)
        model.free()
    finally:
        for t in (tr, tq, tt):
            t.free()


def test_the_combined_configuration_at_small_size(dt):
    """The headline's combination at 60k x 6k: labels from a BF16 search, the
    proposal (M = 1) with BF16 tiles and 512-query blocks; the lists equal the
    plain FP32 search's with 128-query blocks and the oracle's."""
    W = inputs.powerlaw64(n_ref=60_000, n_query=6_000, n_train=6_000)
    tr = dt.dtree_build(torch.from_numpy(W.ref).cuda(), W.leaf_size)
    tq = dt.dtree_build(torch.from_numpy(W.query).cuda(), W.leaf_size)
    tt = dt.dtree_build(torch.from_numpy(W.extra["train"]).cuda(), W.leaf_size)
    try:
        model = dt.dtree_proposal_train(tr, tt, W.k, epochs=5, batch=64, precision="bf16")
        dt.dtree_attach_proposal(tr, model)
        plain = dt.dtree_knn(tq, tr, W.k, precision="fp32", query_block=128)
        idx, dist = dt.dtree_knn(tq, tr, W.k, precision="bf16", proposal=1, query_block=512)
        ti, td = truth(W.ref, W.query, W.k)
        r = compare(idx.cpu().numpy(), dist.cpu().numpy(), ti, td, W.k)
        assert r["exact"] + r["exempt"] == len(W.query)
        assert torch.equal(idx, plain[0])
        dt.dtree_attach_proposal(tr, None)
        model.free()
    finally:
        for t in (tr, tq, tt):
            t.free()
