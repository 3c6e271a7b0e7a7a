"""fp64 reference of the value network -- TEST INFRASTRUCTURE ONLY.

The network that truncates playouts: input x = [P1 stones (cells), P2 stones
(cells), side-to-move (1 when P1 moves)], zero-padded to K columns; two
hidden layers of 512 ReLU units; one tanh output v; the predicted
probability that P1 wins is p = (v + 1) / 2 (a draw counts one half).
Loss: mean squared error between p and the label y (the fraction of random
playouts P1 wins, draws one half).  Optimiser: Adam (Kingma & Ba 2015,
Algorithm 1) with beta1 0.9, beta2 0.999, eps 1e-8, bias-corrected moments.

Everything here is plain fp64 numpy matrix algebra: forward, the chain rule
written out layer by layer, and the Adam update.  The CUDA path keeps its
activations and hidden-layer gradients in bf16; callers compare with a
tolerance derived from that rounding.

Parameter layout (shared with the C-ABI's flat parameter vector):
    W1 [H, K], b1 [H], W2 [H, H], b2 [H], w3 [H], b3 [1]
"""
from __future__ import annotations

import numpy as np

H = 512
BETA1, BETA2, EPS = 0.9, 0.999, 1e-8


def param_shapes(K, hidden=H):
    return [("W1", (hidden, K)), ("b1", (hidden,)), ("W2", (hidden, hidden)), ("b2", (hidden,)),
            ("w3", (hidden,)), ("b3", (1,))]


def num_params(K, hidden=H):
    return sum(int(np.prod(s)) for _, s in param_shapes(K, hidden))


def unflatten(theta, K, hidden=H):
    out, off = {}, 0
    for name, shape in param_shapes(K, hidden):
        n = int(np.prod(shape))
        out[name] = np.asarray(theta[off:off + n], np.float64).reshape(shape)
        off += n
    return out


def flatten(p, K, hidden=H):
    return np.concatenate([np.asarray(p[name], np.float64).reshape(-1) for name, _ in param_shapes(K, hidden)])


def forward(theta, X, K, hidden=H):
    """Returns (p, cache).  X: [B, K] (0/1 inputs)."""
    P = unflatten(theta, K, hidden)
    X = np.asarray(X, np.float64)
    z1 = X @ P["W1"].T + P["b1"]
    h1 = np.maximum(z1, 0.0)
    z2 = h1 @ P["W2"].T + P["b2"]
    h2 = np.maximum(z2, 0.0)
    z3 = h2 @ P["w3"] + P["b3"][0]
    v = np.tanh(z3)
    p = 0.5 * (v + 1.0)
    return p, dict(X=X, z1=z1, h1=h1, z2=z2, h2=h2, v=v, P=P)


def loss(theta, X, y, K, hidden=H):
    p, _ = forward(theta, X, K, hidden)
    return float(np.mean((p - np.asarray(y, np.float64)) ** 2))


def grad(theta, X, y, K, hidden=H):
    """Gradient of `loss` with respect to the flat parameter vector."""
    p, c = forward(theta, X, K, hidden)
    B = p.shape[0]
    P = c["P"]
    dp = 2.0 * (p - np.asarray(y, np.float64)) / B          # dL/dp
    dz3 = dp * 0.5 * (1.0 - c["v"] ** 2)                      # dp/dv = 1/2, dv/dz3 = 1 - v^2
    g = {"w3": c["h2"].T @ dz3, "b3": np.array([dz3.sum()])}
    dh2 = np.outer(dz3, P["w3"])
    dz2 = dh2 * (c["z2"] > 0)
    g["W2"] = dz2.T @ c["h1"]
    g["b2"] = dz2.sum(0)
    dh1 = dz2 @ P["W2"]
    dz1 = dh1 * (c["z1"] > 0)
    g["W1"] = dz1.T @ c["X"]
    g["b1"] = dz1.sum(0)
    return flatten(g, K, hidden)


def adam_step(theta, m, v, g, t, lr):
    """One Adam update at step t (1-based); returns new (theta, m, v)."""
    m = BETA1 * m + (1.0 - BETA1) * g
    v = BETA2 * v + (1.0 - BETA2) * g * g
    mhat = m / (1.0 - BETA1 ** t)
    vhat = v / (1.0 - BETA2 ** t)
    return theta - lr * mhat / (np.sqrt(vhat) + EPS), m, v


def encode(board, to_move, K):
    """Net input rows from canonical boards [B, cells] (0/1/2) and to_move [B]."""
    board = np.asarray(board)
    B, cells = board.shape
    X = np.zeros((B, K), np.float64)
    X[:, :cells] = board == 1
    X[:, cells:2 * cells] = board == 2
    X[:, 2 * cells] = np.asarray(to_move) == 1
    return X


def bf16_round(a):
    """Round-to-nearest-even to bfloat16, returned as float64."""
    a32 = np.asarray(a, np.float32)
    u = a32.view(np.uint32).astype(np.uint64)
    r = ((u + 0x7FFF + ((u >> 16) & 1)) >> 16) << 16
    return r.astype(np.uint32).view(np.float32).astype(np.float64)
