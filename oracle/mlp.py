"""FP64 reference of the cost-model network (test infrastructure only).

x (16) -> h1 = relu(W1 x + b1) -> h2 = relu(W2 h1 + b2) -> y = w3 . h2 + b3,
loss = mean over samples of (y - t)^2, with the parameter vector laid out as
W1[H][16], b1[H], W2[H][H], b2[H], w3[H], b3.  Forward and backward are the
chain rule written out with numpy in float64.
"""
import numpy as np

NIN = 16


def unpack(p, H):
    p = np.asarray(p, dtype=np.float64)
    i = 0
    W1 = p[i:i + H * NIN].reshape(H, NIN)
    i += H * NIN
    b1 = p[i:i + H]
    i += H
    W2 = p[i:i + H * H].reshape(H, H)
    i += H * H
    b2 = p[i:i + H]
    i += H
    w3 = p[i:i + H]
    i += H
    b3 = p[i]
    return W1, b1, W2, b2, w3, b3


def forward(p, X, H):
    W1, b1, W2, b2, w3, b3 = unpack(p, H)
    X = np.asarray(X, dtype=np.float64)
    a1 = X @ W1.T + b1
    h1 = np.maximum(a1, 0.0)
    a2 = h1 @ W2.T + b2
    h2 = np.maximum(a2, 0.0)
    return h2 @ w3 + b3


def loss_and_grad(p, X, T, H):
    W1, b1, W2, b2, w3, b3 = unpack(p, H)
    X = np.asarray(X, dtype=np.float64)
    T = np.asarray(T, dtype=np.float64)
    B = X.shape[0]
    a1 = X @ W1.T + b1
    h1 = np.maximum(a1, 0.0)
    a2 = h1 @ W2.T + b2
    h2 = np.maximum(a2, 0.0)
    y = h2 @ w3 + b3
    r = y - T
    loss = float(np.mean(r * r))
    dy = 2.0 * r / B
    g_w3 = h2.T @ dy
    g_b3 = dy.sum()
    dh2 = np.outer(dy, w3) * (a2 > 0)
    g_W2 = dh2.T @ h1
    g_b2 = dh2.sum(axis=0)
    dh1 = (dh2 @ W2) * (a1 > 0)
    g_W1 = dh1.T @ X
    g_b1 = dh1.sum(axis=0)
    g = np.concatenate([g_W1.ravel(), g_b1, g_W2.ravel(), g_b2, g_w3, [g_b3]])
    return loss, g
