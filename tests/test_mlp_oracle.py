"""Pins of the fp64 value-network oracle (no GPU): its gradient against
central finite differences of its loss, Adam against the update rule worked
by hand for a constant gradient, and the bf16 rounding against values with a
known representation."""
import numpy as np
import pytest

from oracle import mlp as M


def small_problem(K=16, H=8, B=12, seed=0):
    rng = np.random.default_rng(seed)
    theta = np.concatenate([rng.normal(0, 0.5, int(np.prod(s))) for _, s in M.param_shapes(K, H)])
    X = (rng.random((B, K)) < 0.4).astype(np.float64)
    y = rng.random(B)
    return theta, X, y


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_gradient_matches_central_differences(seed):
    K, H = 16, 8
    theta, X, y = small_problem(K, H, seed=seed)
    g = M.grad(theta, X, y, K, H)
    eps = 1e-6
    idx = np.random.default_rng(seed).choice(theta.size, 60, replace=False)
    for i in idx:
        tp, tm = theta.copy(), theta.copy()
        tp[i] += eps
        tm[i] -= eps
        fd = (M.loss(tp, X, y, K, H) - M.loss(tm, X, y, K, H)) / (2 * eps)
        assert abs(fd - g[i]) <= 1e-6 * max(1.0, abs(fd)), (i, fd, g[i])


def test_gradient_every_block_nonzero_and_shapes():
    K, H = 16, 8
    theta, X, y = small_problem(K, H)
    g = M.unflatten(M.grad(theta, X, y, K, H), K, H)
    for name, shape in M.param_shapes(K, H):
        assert g[name].shape == shape
        assert np.abs(g[name]).sum() > 0, name


def test_output_range_and_perfect_prediction_has_zero_loss():
    K, H = 16, 8
    theta, X, _ = small_problem(K, H)
    p, _ = M.forward(theta, X, K, H)
    assert ((p > 0) & (p < 1)).all()
    assert M.loss(theta, X, p, K, H) == 0.0
    assert np.abs(M.grad(theta, X, p, K, H)).max() == 0.0


def test_adam_constant_gradient_closed_form():
    # With a constant gradient g, the bias-corrected moments are exactly
    # m_hat = g and v_hat = g^2 at every step, so each step moves the
    # parameter by lr * g / (|g| + eps).
    g = np.array([0.5, -2.0, 1e-3])
    th, m, v = np.zeros(3), np.zeros(3), np.zeros(3)
    lr = 1e-3
    for t in range(1, 6):
        th, m, v = M.adam_step(th, m, v, g, t, lr)
        want = -t * lr * g / (np.abs(g) + M.EPS)
        assert np.allclose(th, want, rtol=1e-12, atol=1e-15)


def test_encode_layout():
    board = np.array([[0, 1, 2, 1], [2, 0, 0, 0]], np.int8)
    X = M.encode(board, np.array([1, 2]), 12)
    assert X[0].tolist() == [0, 1, 0, 1, 0, 0, 1, 0, 1, 0, 0, 0]
    assert X[1].tolist() == [0, 0, 0, 0, 1, 0, 0, 0, 0, 0, 0, 0]


def test_bf16_round_known_values():
    assert M.bf16_round(1.0) == 1.0
    assert M.bf16_round(1.0 + 2 ** -8) == 1.0               # tie: rounds to even
    assert M.bf16_round(1.0 + 3 * 2 ** -8) == 1.0 + 2 ** -6  # tie: rounds up to even
    assert M.bf16_round(1.0 + 2 ** -7) == 1.0 + 2 ** -7      # representable
    assert M.bf16_round(-3.0) == -3.0
    x = np.random.default_rng(0).normal(size=1000)
    r = M.bf16_round(x)
    assert np.all(np.abs(r - x) <= np.abs(x) * 2 ** -8)
