"""FP64 reference of the learned rank proposal's network -- test infrastructure only.

Only the tests, the package's smoke check and the benchmark's CPU baseline use this module;
the library never calls it.

The network maps the 12 features of a far block's sum-expression to a prediction of
log2(1 + eps-rank) of the block (the rank a compression of Algorithm 8 ends at):

    h1 = relu(W1 x + b1)      W1: 64 x 12
    h2 = relu(W2 h1 + b2)     W2: 64 x 64
    y  = w3 . h2 + b3

and the training loss over a batch is the mean squared error mean_s (y_s - t_s)^2. Parameters are
one flat vector: W1 (row-major, W1[j][i] at j*12 + i), b1, W2 (row-major), b2, w3, b3 -- 5057
numbers. The gradient is the chain rule written out layer by layer, in FP64.

Pins (tests/test_oracle.py): central finite differences of loss(); a network with zero weights
(output = b3, closed-form gradient); a network whose pre-activations are all positive (then it is
the affine map W3 W2 W1 x + ..., computed by plain matrix products).
"""
from __future__ import annotations

import numpy as np

F, H = 12, 64
N_PARAMS = H * F + H + H * H + H + H + 1


def unpack(w: np.ndarray):
    """(W1, b1, W2, b2, w3, b3) views of the flat parameter vector."""
    w = np.asarray(w, np.float64)
    assert w.shape == (N_PARAMS,)
    o = 0
    W1 = w[o:o + H * F].reshape(H, F); o += H * F
    b1 = w[o:o + H]; o += H
    W2 = w[o:o + H * H].reshape(H, H); o += H * H
    b2 = w[o:o + H]; o += H
    w3 = w[o:o + H]; o += H
    b3 = w[o]
    return W1, b1, W2, b2, w3, b3


def forward(w: np.ndarray, X: np.ndarray) -> np.ndarray:
    """Network output y for each row of X (count x 12), FP64."""
    W1, b1, W2, b2, w3, b3 = unpack(w)
    X = np.asarray(X, np.float64)
    h1 = np.maximum(X @ W1.T + b1, 0.0)
    h2 = np.maximum(h1 @ W2.T + b2, 0.0)
    return h2 @ w3 + b3


def loss(w: np.ndarray, X: np.ndarray, t: np.ndarray) -> float:
    """Mean squared error of the network on targets t."""
    e = forward(w, X) - np.asarray(t, np.float64)
    return float(np.mean(e * e))


def loss_grad(w: np.ndarray, X: np.ndarray, t: np.ndarray):
    """(loss, gradient of the loss with respect to the flat parameters), FP64 backpropagation."""
    W1, b1, W2, b2, w3, b3 = unpack(w)
    X = np.asarray(X, np.float64)
    t = np.asarray(t, np.float64)
    count = X.shape[0]
    a1 = X @ W1.T + b1
    h1 = np.maximum(a1, 0.0)
    a2 = h1 @ W2.T + b2
    h2 = np.maximum(a2, 0.0)
    y = h2 @ w3 + b3
    e = y - t
    dy = 2.0 * e / count                       # d loss / d y_s
    g_b3 = dy.sum()
    g_w3 = h2.T @ dy
    da2 = np.outer(dy, w3) * (a2 > 0.0)        # d loss / d a2
    g_W2 = da2.T @ h1
    g_b2 = da2.sum(axis=0)
    da1 = (da2 @ W2) * (a1 > 0.0)
    g_W1 = da1.T @ X
    g_b1 = da1.sum(axis=0)
    g = np.concatenate([g_W1.ravel(), g_b1, g_W2.ravel(), g_b2, g_w3, [g_b3]])
    return float(np.mean(e * e)), g


def target(ranks: np.ndarray) -> np.ndarray:
    """Training target of a rank: log2(1 + rank)."""
    return np.log2(1.0 + np.maximum(np.asarray(ranks, np.float64), 0.0))


def predicted_rank(y: np.ndarray) -> np.ndarray:
    """Inverse of target(), clipped at zero."""
    return np.maximum(np.exp2(np.asarray(y, np.float64)) - 1.0, 0.0)
