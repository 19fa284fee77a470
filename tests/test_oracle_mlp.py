"""Pins of the FP64 selector-network oracle: central finite differences, a
closed-form case, and the first Adam step in closed form (CPU only)."""
import numpy as np

from oracle import mlp


def _rand_theta(seed, scale=0.3):
    return np.random.default_rng(seed).standard_normal(mlp.N_PARAMS) * scale


def test_param_count_and_layout():
    assert mlp.N_PARAMS == 8 * 64 + 64 + 64 * 64 + 64 + 2 * 64 + 2 == 4866
    th = np.arange(mlp.N_PARAMS, dtype=np.float64)
    p = mlp.unpack(th)
    assert p["W1"][0, 1] == 1 and p["b1"][0] == 512 and p["W2"][0, 0] == 576
    assert p["b3"][1] == mlp.N_PARAMS - 1
    assert np.array_equal(mlp.pack(p), th)


def test_gradient_matches_central_differences():
    rng = np.random.default_rng(1)
    X = rng.standard_normal((16, 8))
    T = rng.standard_normal((16, 2))
    th = _rand_theta(2)
    L, g = mlp.grad(th, X, T)
    assert abs(L - mlp.loss(th, X, T)) < 1e-12
    h = 1e-6
    idx = rng.choice(mlp.N_PARAMS, 300, replace=False)
    for k in idx:
        e = np.zeros_like(th)
        e[k] = h
        fd = (mlp.loss(th + e, X, T) - mlp.loss(th - e, X, T)) / (2 * h)
        assert abs(fd - g[k]) <= 1e-6 * max(1.0, abs(fd)), k


def test_closed_form_zero_hidden_weights():
    """W1 = 0, b1 = 0 => A1 = 0, A2 = relu(b2), Y = W3 relu(b2) + b3 for every
    row; the gradients of the output layer are then closed forms."""
    rng = np.random.default_rng(3)
    p = mlp.unpack(_rand_theta(4))
    p = {k: v.copy() for k, v in p.items()}
    p["W1"][:] = 0.0
    p["b1"][:] = 0.0
    th = mlp.pack(p)
    X = rng.standard_normal((10, 8))
    T = rng.standard_normal((10, 2))
    a2 = np.maximum(p["b2"], 0.0)
    y = p["W3"] @ a2 + p["b3"]
    Y, _ = mlp.forward(th, X)
    assert np.allclose(Y, y[None, :], atol=1e-14)
    L, g = mlp.grad(th, X, T)
    r = (y[None, :] - T)                       # [10][2]
    gb3 = 2.0 * r.sum(0) / r.size
    gW3 = np.outer(gb3, a2)
    G = mlp.unpack(g)
    assert np.allclose(G["b3"], gb3, atol=1e-14)
    assert np.allclose(G["W3"], gW3, atol=1e-14)
    # no signal reaches W1 through a zero hidden layer (ReLU'(0) = 0 here)
    assert np.all(G["W1"] == 0.0)


def test_adam_first_step_closed_form():
    th = _rand_theta(5)
    g = np.random.default_rng(6).standard_normal(mlp.N_PARAMS)
    m = np.zeros_like(th)
    v = np.zeros_like(th)
    th1, m1, v1 = mlp.adam(th, g, m, v, 1, lr=1e-3)
    # bias-corrected first step: lr * g / (|g| + eps)
    assert np.allclose(th - th1, 1e-3 * g / (np.abs(g) + 1e-8), rtol=1e-12)
    assert np.allclose(m1, 0.1 * g) and np.allclose(v1, 0.001 * g * g)


def test_training_reduces_loss_on_linear_target():
    rng = np.random.default_rng(8)
    X = rng.standard_normal((256, 8))
    w = rng.standard_normal((8, 2))
    T = X @ w
    th = _rand_theta(9, 0.2)
    m = np.zeros_like(th)
    v = np.zeros_like(th)
    L0 = mlp.loss(th, X, T)
    for t in range(1, 301):
        _, g = mlp.grad(th, X, T)
        th, m, v = mlp.adam(th, g, m, v, t, lr=3e-3)
    assert mlp.loss(th, X, T) < 0.1 * L0
