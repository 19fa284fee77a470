"""FP64 oracle of the repair-strategy selector network (test infrastructure only).

The paper has no learned component; the selector is the build's own addition
that picks incremental repair or rebuild per step.  Its behaviour is fixed here:

* network 8 -> 64 -> 64 -> 2, ReLU after each hidden layer, linear output
  (outputs: predicted ln step time of incremental repair, of rebuild);
* loss = mean over the batch and both outputs of (y - t)^2;
* Adam with bias correction.

Flat parameter layout (shared interface with the GPU trainer, float32 there):
``W1[64][8], b1[64], W2[64][64], b2[64], W3[2][64], b3[2]`` -- 4866 values.

Written as the textbook forward / reverse-mode chain rule in plain numpy
float64; pinned by central finite differences and a closed-form case in
``tests/test_oracle_mlp.py``.
"""
from __future__ import annotations

import numpy as np

D_IN, D_H, D_OUT = 8, 64, 2
SHAPES = [("W1", (D_H, D_IN)), ("b1", (D_H,)), ("W2", (D_H, D_H)), ("b2", (D_H,)),
          ("W3", (D_OUT, D_H)), ("b3", (D_OUT,))]
N_PARAMS = sum(int(np.prod(s)) for _, s in SHAPES)


def unpack(theta):
    theta = np.asarray(theta, np.float64)
    assert theta.shape == (N_PARAMS,)
    out, k = {}, 0
    for name, shp in SHAPES:
        sz = int(np.prod(shp))
        out[name] = theta[k:k + sz].reshape(shp)
        k += sz
    return out


def pack(p) -> np.ndarray:
    return np.concatenate([np.asarray(p[name], np.float64).ravel() for name, _ in SHAPES])


def forward(theta, X):
    """Returns (Y, cache). X: [B][8]."""
    p = unpack(theta)
    X = np.asarray(X, np.float64)
    Z1 = X @ p["W1"].T + p["b1"]
    A1 = np.maximum(Z1, 0.0)
    Z2 = A1 @ p["W2"].T + p["b2"]
    A2 = np.maximum(Z2, 0.0)
    Y = A2 @ p["W3"].T + p["b3"]
    return Y, (X, Z1, A1, Z2, A2)


def loss(theta, X, T) -> float:
    Y, _ = forward(theta, X)
    return float(np.mean((Y - np.asarray(T, np.float64)) ** 2))


def grad(theta, X, T):
    """(loss, dloss/dtheta) by the chain rule, in the flat layout."""
    p = unpack(theta)
    Y, (X, Z1, A1, Z2, A2) = forward(theta, X)
    T = np.asarray(T, np.float64)
    n = Y.size
    dY = 2.0 * (Y - T) / n
    g = {}
    g["W3"] = dY.T @ A2
    g["b3"] = dY.sum(axis=0)
    dA2 = dY @ p["W3"]
    dZ2 = dA2 * (Z2 > 0)
    g["W2"] = dZ2.T @ A1
    g["b2"] = dZ2.sum(axis=0)
    dA1 = dZ2 @ p["W2"]
    dZ1 = dA1 * (Z1 > 0)
    g["W1"] = dZ1.T @ X
    g["b1"] = dZ1.sum(axis=0)
    return float(np.mean((Y - T) ** 2)), pack(g)


def adam(theta, g, m, v, t: int, lr=1e-3, beta1=0.9, beta2=0.999, eps=1e-8):
    """One Adam update (Kingma & Ba, Algorithm 1); t counts from 1."""
    m = beta1 * m + (1.0 - beta1) * g
    v = beta2 * v + (1.0 - beta2) * g * g
    mh = m / (1.0 - beta1 ** t)
    vh = v / (1.0 - beta2 ** t)
    return theta - lr * mh / (np.sqrt(vh) + eps), m, v
