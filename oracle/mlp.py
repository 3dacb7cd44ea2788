"""Plain numpy reference of the autotuner's cost-model network (test
infrastructure only; the product trains it with its own CUDA kernels).

The paper has no learned component; this is the CPU oracle the GPU forward
and backward passes are checked against.  Network: x -> tanh(W1 x + b1) ->
tanh(W2 h1 + b2) -> y = w3 . h2 + b3, loss = mean over the batch of
(y - t)^2.  Parameters in one flat vector, in the order W1 [n_h][n_in], b1,
W2 [n_h][n_h], b2, w3 [n_h], b3.  All arithmetic in float64.
"""
from __future__ import annotations

import numpy as np


def unpack(p, n_in, n_h):
    p = np.asarray(p, dtype=np.float64)
    i = 0
    W1 = p[i:i + n_h * n_in].reshape(n_h, n_in); i += n_h * n_in
    b1 = p[i:i + n_h]; i += n_h
    W2 = p[i:i + n_h * n_h].reshape(n_h, n_h); i += n_h * n_h
    b2 = p[i:i + n_h]; i += n_h
    w3 = p[i:i + n_h]; i += n_h
    b3 = p[i]; i += 1
    assert i == p.size
    return W1, b1, W2, b2, w3, b3


def num_params(n_in, n_h):
    return n_h * n_in + n_h + n_h * n_h + n_h + n_h + 1


def forward(p, X, n_in, n_h):
    W1, b1, W2, b2, w3, b3 = unpack(p, n_in, n_h)
    X = np.asarray(X, dtype=np.float64)
    H1 = np.tanh(X @ W1.T + b1)
    H2 = np.tanh(H1 @ W2.T + b2)
    return H2 @ w3 + b3, (H1, H2)


def loss_and_gradient(p, X, T, n_in, n_h):
    """Mean squared error and its gradient by the chain rule (backprop)."""
    W1, b1, W2, b2, w3, b3 = unpack(p, n_in, n_h)
    X = np.asarray(X, dtype=np.float64)
    T = np.asarray(T, dtype=np.float64)
    B = X.shape[0]
    y, (H1, H2) = forward(p, X, n_in, n_h)
    dy = 2.0 * (y - T) / B
    g_w3 = H2.T @ dy
    g_b3 = dy.sum()
    dA2 = np.outer(dy, w3) * (1.0 - H2 ** 2)
    g_W2 = dA2.T @ H1
    g_b2 = dA2.sum(0)
    dA1 = (dA2 @ W2) * (1.0 - H1 ** 2)
    g_W1 = dA1.T @ X
    g_b1 = dA1.sum(0)
    g = np.concatenate([g_W1.ravel(), g_b1, g_W2.ravel(), g_b2, g_w3, [g_b3]])
    return float(np.mean((y - T) ** 2)), g
