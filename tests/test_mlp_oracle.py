"""Pins of the fp64 cost-model reference (oracle/mlp_ref.py): a hand-set net
with a closed-form output, central finite differences of the loss, the
closed form of Adam's first step, and loss reduction on a target the net can
represent."""
import numpy as np

from oracle import mlp_ref


def test_hand_set_net_closed_form():
    # F = 2, H = 2: h1 = relu(x), h2 = h1, y = h2[0] - h2[1] + 0.5
    p = mlp_ref.pack(np.eye(2), np.zeros(2), np.eye(2), np.zeros(2), np.array([1.0, -1.0]), np.array([0.5]))
    X = np.array([[3.0, 1.0], [-2.0, 4.0], [2.0, -7.0], [0.0, 0.0]])
    y, _ = mlp_ref.forward(p, X, np.zeros(2), np.ones(2), 2)
    assert np.allclose(y, [2.5, -3.5, 2.5, 0.5])
    # standardisation: (x - mu) / sigma before the first layer
    y2, _ = mlp_ref.forward(p, X * 2 + 1, np.ones(2), np.full(2, 2.0), 2)
    assert np.allclose(y2, y)


def test_backward_matches_central_differences():
    rng = np.random.default_rng(0)
    F, H, B = 5, 8, 7
    p = mlp_ref.init(F, H, seed=1) + rng.normal(0, 0.05, mlp_ref.n_params(F, H))
    X = rng.normal(size=(B, F))
    t = rng.normal(size=B)
    mu, sigma = X.mean(0), X.std(0) + 0.1
    y, cache = mlp_ref.forward(p, X, mu, sigma, H)
    g = mlp_ref.backward(p, cache, y, t, H)
    eps = 1e-6
    num = np.empty_like(p)
    for i in range(len(p)):
        d = np.zeros_like(p)
        d[i] = eps
        lp = mlp_ref.loss(mlp_ref.forward(p + d, X, mu, sigma, H)[0], t)
        lm = mlp_ref.loss(mlp_ref.forward(p - d, X, mu, sigma, H)[0], t)
        num[i] = (lp - lm) / (2 * eps)
    assert np.allclose(g, num, rtol=1e-5, atol=1e-8)


def test_adam_first_step_moves_each_parameter_by_lr():
    # k = 1: m_hat = g and v_hat = g^2, so the step is lr * g / (|g| + eps)
    p = np.array([1.0, -2.0, 0.5, 3.0])
    g = np.array([0.3, -4.0, 1e-3, -2.0])
    p1, m, v = mlp_ref.adam_step(p, g, np.zeros(4), np.zeros(4), 1, lr=0.01, eps=1e-12)
    assert np.allclose(p1, p - 0.01 * np.sign(g), atol=1e-9)
    assert np.allclose(m, 0.1 * g) and np.allclose(v, 0.001 * g * g)


def test_training_reduces_loss_on_a_representable_target():
    rng = np.random.default_rng(3)
    F, H, B = 6, 16, 256
    X = rng.normal(size=(B, F))
    t = np.maximum(X @ rng.normal(size=F), 0.0) - 0.5 * X[:, 0]  # a small relu net fits it
    mu, sigma = X.mean(0), X.std(0)
    p = mlp_ref.init(F, H, seed=4)
    m = np.zeros_like(p)
    v = np.zeros_like(p)
    y, cache = mlp_ref.forward(p, X, mu, sigma, H)
    l0 = mlp_ref.loss(y, t)
    for k in range(1, 601):
        y, cache = mlp_ref.forward(p, X, mu, sigma, H)
        p, m, v = mlp_ref.adam_step(p, mlp_ref.backward(p, cache, y, t, H), m, v, k, lr=3e-3)
    assert mlp_ref.loss(mlp_ref.forward(p, X, mu, sigma, H)[0], t) < 0.02 * l0
