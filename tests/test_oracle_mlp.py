"""Pins of the FP64 cost-model network oracle (CPU only): a hand-computed
one-unit network, the all-zero network, and central finite differences of
its loss against its backward pass."""
import numpy as np

from oracle import mlp


def test_hand_computed_one_unit():
    H = 1
    W1 = np.zeros((1, 16))
    W1[0, 0], W1[0, 3] = 2.0, -1.0
    b1 = np.array([0.5])
    W2 = np.array([[3.0]])
    b2 = np.array([-1.0])
    w3 = np.array([0.25])
    b3 = 0.1
    p = np.concatenate([W1.ravel(), b1, W2.ravel(), b2, w3, [b3]])
    x = np.zeros((2, 16))
    x[0, 0], x[0, 3] = 1.0, 0.5      # a1 = 2 - 0.5 + 0.5 = 2 -> h1 = 2 -> a2 = 5 -> y = 1.35
    x[1, 0], x[1, 3] = -1.0, 1.0     # a1 = -2.5 -> h1 = 0 -> a2 = -1 -> h2 = 0 -> y = 0.1
    y = mlp.forward(p, x, H)
    np.testing.assert_allclose(y, [1.35, 0.1], atol=1e-15)


def test_zero_network():
    H = 4
    P = H * 16 + H + H * H + H + H + 1
    p = np.zeros(P)
    p[-1] = 0.7
    X = np.random.default_rng(0).normal(size=(5, 16))
    T = np.arange(5.0)
    loss, g = mlp.loss_and_grad(p, X, T, H)
    assert abs(loss - np.mean((0.7 - T) ** 2)) < 1e-15
    assert abs(g[-1] - np.mean(2 * (0.7 - T))) < 1e-15
    assert np.all(g[:-1] == 0)


def test_backward_matches_finite_differences():
    H = 6
    P = H * 16 + H + H * H + H + H + 1
    rng = np.random.default_rng(1)
    p = rng.normal(scale=0.5, size=P)
    X = rng.normal(size=(9, 16))
    T = rng.normal(size=9)
    _, g = mlp.loss_and_grad(p, X, T, H)
    eps = 1e-6
    fd = np.zeros(P)
    for i in range(P):
        e = np.zeros(P)
        e[i] = eps
        fd[i] = (mlp.loss_and_grad(p + e, X, T, H)[0] - mlp.loss_and_grad(p - e, X, T, H)[0]) / (2 * eps)
    np.testing.assert_allclose(g, fd, atol=1e-7, rtol=1e-6)
