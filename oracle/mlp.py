"""FP64 reference of the learned proposal's network (test infrastructure).

Only the tests may import this module: it is the oracle the GPU's forward
and backward kernels are checked against, never a fallback for them.

The network maps x (d) to logits z (C) through two hidden ReLU layers of
width 256:
    h1 = relu(W1 x + b1),  h2 = relu(W2 h1 + b2),  z = W3 h2 + b3,
and the loss of a batch of n rows against target distributions t (rows
summing to 1) is the mean softmax cross-entropy
    L = (1/n) sum_rows -sum_c t_c log softmax(z)_c.
The gradients below are the chain rule written out layer by layer; they are
pinned by central finite differences in the tests.
"""
from __future__ import annotations

from typing import Dict, Sequence, Tuple

import numpy as np

NAMES = ("W1", "b1", "W2", "b2", "W3", "b3")


def init(d: int, C: int, H: int = 256, seed: int = 0, scale: float = 1.0) -> Dict[str, np.ndarray]:
    """Random float64 parameters (He-uniform weights times `scale`, small biases)."""
    g = np.random.default_rng(seed)
    def w(o, i):
        lim = np.sqrt(6.0 / i) * scale
        return g.uniform(-lim, lim, size=(o, i))
    return {"W1": w(H, d), "b1": g.uniform(-0.1, 0.1, H), "W2": w(H, H),
            "b2": g.uniform(-0.1, 0.1, H), "W3": w(C, H), "b3": g.uniform(-0.1, 0.1, C)}


def forward(p: Dict[str, np.ndarray], X: np.ndarray) -> Tuple[np.ndarray, ...]:
    X = np.asarray(X, dtype=np.float64)
    a1 = X @ p["W1"].T + p["b1"]
    h1 = np.maximum(a1, 0.0)
    a2 = h1 @ p["W2"].T + p["b2"]
    h2 = np.maximum(a2, 0.0)
    z = h2 @ p["W3"].T + p["b3"]
    return a1, h1, a2, h2, z


def log_softmax(z: np.ndarray) -> np.ndarray:
    m = z.max(axis=1, keepdims=True)
    return z - m - np.log(np.exp(z - m).sum(axis=1, keepdims=True))


def loss(p: Dict[str, np.ndarray], X: np.ndarray, T: np.ndarray) -> float:
    z = forward(p, X)[-1]
    return float(-(np.asarray(T, dtype=np.float64) * log_softmax(z)).sum() / X.shape[0])


def loss_grad(p: Dict[str, np.ndarray], X: np.ndarray, T: np.ndarray):
    """(loss, gradients) of the mean softmax cross-entropy."""
    X = np.asarray(X, dtype=np.float64)
    T = np.asarray(T, dtype=np.float64)
    n = X.shape[0]
    a1, h1, a2, h2, z = forward(p, X)
    ls = log_softmax(z)
    L = float(-(T * ls).sum() / n)
    dz = (np.exp(ls) - T) / n                 # d L / d z
    g = {"W3": dz.T @ h2, "b3": dz.sum(axis=0)}
    dh2 = dz @ p["W3"]
    da2 = dh2 * (a2 > 0)                       # ReLU'
    g["W2"] = da2.T @ h1
    g["b2"] = da2.sum(axis=0)
    dh1 = da2 @ p["W2"]
    da1 = dh1 * (a1 > 0)
    g["W1"] = da1.T @ X
    g["b1"] = da1.sum(axis=0)
    return L, g


def finite_difference(p: Dict[str, np.ndarray], X: np.ndarray, T: np.ndarray, name: str,
                      entries: Sequence[Tuple[int, ...]], h: float = 1e-6) -> np.ndarray:
    """Central differences of the loss in the given entries of one parameter."""
    out = []
    for ix in entries:
        q = {k: v.copy() for k, v in p.items()}
        q[name][ix] += h
        up = loss(q, X, T)
        q[name][ix] -= 2 * h
        dn = loss(q, X, T)
        out.append((up - dn) / (2 * h))
    return np.array(out)
