"""Pins of the FP64 proposal-network oracle (no GPU): its gradients against
central finite differences, and closed forms of the loss."""
import numpy as np
import pytest

from oracle import mlp


def _batch(n=7, d=5, C=11, seed=3):
    g = np.random.default_rng(seed)
    X = g.normal(size=(n, d))
    T = g.random(size=(n, C))
    T[:, ::3] = 0.0
    T /= T.sum(axis=1, keepdims=True)
    return X, T


@pytest.mark.parametrize("name", mlp.NAMES)
def test_gradients_match_finite_differences(name):
    X, T = _batch()
    p = mlp.init(5, 11, H=256, seed=1)
    _, g = mlp.loss_grad(p, X, T)
    rng = np.random.default_rng(7)
    shape = p[name].shape
    entries = [tuple(int(rng.integers(0, s)) for s in shape) for _ in range(12)]
    fd = mlp.finite_difference(p, X, T, name, entries)
    an = np.array([g[name][ix] for ix in entries])
    assert np.allclose(an, fd, rtol=1e-5, atol=1e-9), (an, fd)


def test_uniform_logits_give_log_C():
    # zero output weights and bias: every class is equally likely
    X, T = _batch(C=13)
    p = mlp.init(5, 13, seed=2)
    p["W3"][:] = 0.0
    p["b3"][:] = 0.0
    assert mlp.loss(p, X, T) == pytest.approx(np.log(13.0), rel=1e-12)


def test_one_hot_target_is_negative_log_probability():
    X, _ = _batch(n=1, C=4)
    p = mlp.init(5, 4, seed=4)
    z = mlp.forward(p, X)[-1][0]
    for c in range(4):
        T = np.zeros((1, 4))
        T[0, c] = 1.0
        ref = -(z[c] - np.log(np.exp(z).sum()))
        assert mlp.loss(p, X, T) == pytest.approx(ref, rel=1e-12)


def test_logit_shift_invariance_and_zero_gradient_at_the_softmax():
    X, T = _batch()
    p = mlp.init(5, 11, seed=5)
    q = {k: v.copy() for k, v in p.items()}
    q["b3"] += 17.0  # softmax ignores a constant added to every logit
    assert mlp.loss(p, X, T) == pytest.approx(mlp.loss(q, X, T), rel=1e-12)
    # targets equal to the model's own softmax: the output gradient vanishes
    z = mlp.forward(p, X)[-1]
    P = np.exp(mlp.log_softmax(z))
    _, g = mlp.loss_grad(p, X, P)
    assert np.abs(g["b3"]).max() < 1e-15 and np.abs(g["W3"]).max() < 1e-14


def test_dead_relu_units_get_no_gradient():
    X, T = _batch()
    p = mlp.init(5, 11, seed=6)
    p["b1"][:5] = -1e6  # these hidden units never fire
    _, g = mlp.loss_grad(p, X, T)
    assert np.all(g["W1"][:5] == 0.0) and np.all(g["b1"][:5] == 0.0)
