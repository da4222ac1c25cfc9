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


def _hand_network():
    """A 2 -> 2 -> 2 -> 2 network whose every value is worked out by hand.

    W1 = [[1, 0], [-1, 1]], b1 = [0.5, 0.5]
    W2 = [[1, 2], [-1, 1]], b2 = [-0.5, 0.25]
    W3 = [[1, -1], [0.5, 3]], b3 = [0, -1]

    row x = (2, 1):
      a1 = (2 + 0.5, -2 + 1 + 0.5)           = (2.5, -0.5)   h1 = (2.5, 0)
      a2 = (2.5 + 0 - 0.5, -2.5 + 0 + 0.25)  = (2, -2.25)    h2 = (2, 0)
      z  = (2 - 0 + 0, 1 + 0 - 1)            = (2, 0)
    row x = (-1, 3):
      a1 = (-1 + 0.5, 1 + 3 + 0.5)           = (-0.5, 4.5)   h1 = (0, 4.5)
      a2 = (0 + 9 - 0.5, 0 + 4.5 + 0.25)     = (8.5, 4.75)   h2 = (8.5, 4.75)
      z  = (8.5 - 4.75 + 0, 4.25 + 14.25 - 1) = (3.75, 17.5)

    Each ReLU zeroes a negative pre-activation in one row and passes a
    positive one in the other, the weights are not symmetric and d = H, so a
    dropped ReLU, a dropped bias, a transposed weight or layers 1 and 2
    applied in the other order all change z (e.g. without the second ReLU
    the first row's z is (4.25, -6.75); with the layers swapped it is (4, 1)).
    """
    p = {"W1": np.array([[1.0, 0.0], [-1.0, 1.0]]), "b1": np.array([0.5, 0.5]),
         "W2": np.array([[1.0, 2.0], [-1.0, 1.0]]), "b2": np.array([-0.5, 0.25]),
         "W3": np.array([[1.0, -1.0], [0.5, 3.0]]), "b3": np.array([0.0, -1.0])}
    X = np.array([[2.0, 1.0], [-1.0, 3.0]])
    return p, X


def test_forward_matches_a_hand_computed_network():
    p, X = _hand_network()
    assert set(mlp.init(d=2, C=2, H=2)) == set(p)  # the parameter set the oracle expects
    a1, h1, a2, h2, z = mlp.forward(p, X)
    # every value is a short binary fraction, so float64 holds it exactly
    assert np.array_equal(a1, [[2.5, -0.5], [-0.5, 4.5]])
    assert np.array_equal(h1, [[2.5, 0.0], [0.0, 4.5]])
    assert np.array_equal(a2, [[2.0, -2.25], [8.5, 4.75]])
    assert np.array_equal(h2, [[2.0, 0.0], [8.5, 4.75]])
    assert np.array_equal(z, [[2.0, 0.0], [3.75, 17.5]])


def test_loss_of_the_hand_computed_network():
    import math

    p, X = _hand_network()
    T = np.array([[1.0, 0.0], [0.25, 0.75]])
    # row 1: z = (2, 0), target class 0: -log p0 = log(1 + e^-2)
    # row 2: z = (3.75, 17.5): -log p1 = log(1 + e^-13.75), -log p0 = 13.75 + log(1 + e^-13.75)
    r1 = math.log1p(math.exp(-2.0))
    r2 = 0.25 * (13.75 + math.log1p(math.exp(-13.75))) + 0.75 * math.log1p(math.exp(-13.75))
    assert mlp.loss(p, X, T) == pytest.approx((r1 + r2) / 2.0, rel=1e-14)
    # the output-layer gradient by hand: dL/dz = (softmax(z) - T) / n
    L, g = mlp.loss_grad(p, X, T)
    s1 = 1.0 / (1.0 + math.exp(-2.0))          # softmax(z_row1)[0]
    s2 = 1.0 / (1.0 + math.exp(13.75))         # softmax(z_row2)[0]
    dz = np.array([[s1 - 1.0, (1.0 - s1) - 0.0], [s2 - 0.25, (1.0 - s2) - 0.75]]) / 2.0
    assert np.allclose(g["b3"], dz.sum(axis=0), rtol=1e-12, atol=1e-15)
    # W3's gradient is dz^T h2 with h2 = [[2, 0], [8.5, 4.75]]
    assert np.allclose(g["W3"], dz.T @ np.array([[2.0, 0.0], [8.5, 4.75]]), rtol=1e-12, atol=1e-15)
