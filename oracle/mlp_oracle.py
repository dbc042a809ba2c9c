"""FP64 reference of the elimination-order ranker's network.

TEST INFRASTRUCTURE ONLY: used by tests/ to check the CUDA forward, backward and
Adam kernels; never imported by the library.

The network is the plain definition: x (F inputs) -> h1 = relu(W1 x + b1) ->
h2 = relu(W2 h1 + b2) -> y = w3 . h2 + b3, with the loss L = mean_r (y_r - t_r)^2.
Its gradient is the chain rule written out layer by layer (relu'(a) = 1 for
a > 0, else 0).  Adam is Kingma and Ba's update with bias correction.
Parameters are one vector [W1 (H x F, row-major), b1, W2 (H x H), b2, w3, b3],
the layout of the library's parameter array.  The pins (finite differences, a
closed form at a degenerate point, the first Adam step) are in
tests/test_oracle_mlp.py.
"""
import numpy as np


def param_count(F, H):
    return H * F + H + H * H + H + H + 1


def unpack(params, F, H):
    p = np.asarray(params, dtype=np.float64)
    assert p.size == param_count(F, H)
    i = 0
    W1 = p[i:i + H * F].reshape(H, F); i += H * F
    b1 = p[i:i + H]; i += H
    W2 = p[i:i + H * H].reshape(H, H); i += H * H
    b2 = p[i:i + H]; i += H
    w3 = p[i:i + H]; i += H
    b3 = p[i]
    return W1, b1, W2, b2, w3, b3


def pack(W1, b1, W2, b2, w3, b3):
    return np.concatenate([W1.ravel(), b1, W2.ravel(), b2, w3, [b3]])


def forward(params, F, H, X):
    W1, b1, W2, b2, w3, b3 = unpack(params, F, H)
    X = np.asarray(X, dtype=np.float64)
    a1 = X @ W1.T + b1
    h1 = np.maximum(a1, 0.0)
    a2 = h1 @ W2.T + b2
    h2 = np.maximum(a2, 0.0)
    y = h2 @ w3 + b3
    return y, (X, a1, h1, a2, h2)


def loss_and_grad(params, F, H, X, t):
    W1, b1, W2, b2, w3, b3 = unpack(params, F, H)
    y, (X, a1, h1, a2, h2) = forward(params, F, H, X)
    R = X.shape[0]
    e = y - np.asarray(t, dtype=np.float64)
    loss = float(np.mean(e * e))
    dy = 2.0 * e / R                               # dL/dy_r
    dw3 = h2.T @ dy
    db3 = dy.sum()
    g2 = np.outer(dy, w3) * (a2 > 0)              # dL/da2
    dW2 = g2.T @ h1
    db2 = g2.sum(axis=0)
    g1 = (g2 @ W2) * (a1 > 0)                     # dL/da1
    dW1 = g1.T @ X
    db1 = g1.sum(axis=0)
    return loss, pack(dW1, db1, dW2, db2, dw3, db3)


def adam(params, grad, m, v, step, lr, beta1, beta2, eps):
    """One Adam step at step number `step` >= 1; returns (params, m, v)."""
    m = beta1 * m + (1.0 - beta1) * grad
    v = beta2 * v + (1.0 - beta2) * grad * grad
    mh = m / (1.0 - beta1 ** step)
    vh = v / (1.0 - beta2 ** step)
    return params - lr * mh / (np.sqrt(vh) + eps), m, v
