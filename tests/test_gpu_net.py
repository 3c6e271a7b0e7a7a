"""GPU parity of the value network kernels against the fp64 oracle.

Tolerances follow from the precision the kernels use: BF16 weights, BF16
hidden activations and hidden-layer gradients (unit roundoff 2^-8), FP32
accumulation.  Against an fp64 evaluation that applies the same BF16
rounding to weights and activations, outputs agree to ~1e-4; against the
plain fp64 definition the gradients agree to a few percent.
"""
import numpy as np
import pytest
import torch

from oracle import games as G
from oracle import mlp as M
from paper_2506_22609_b300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def L(cuda_device):
    from paper_2506_22609_b300 import build

    build.build()
    from paper_2506_22609_b300 import ludax

    ludax.lib()
    return ludax


def bf16_bits(x):
    """float array -> int16 tensor holding bf16 bits (round to nearest even)."""
    t = torch.from_numpy(np.asarray(x, np.float32))
    return t.to(torch.bfloat16).view(torch.int16).cuda()


def rounded_theta(theta, K):
    """Weights rounded to bf16 as the GEMMs see them; biases stay fp32."""
    P = M.unflatten(theta, K)
    for k in ("W1", "W2", "w3"):
        P[k] = M.bf16_round(P[k])
    return M.flatten(P, K)


def forward_bf16(theta, X, K):
    """fp64 forward with the kernels' rounding points (bf16 weights and hidden activations)."""
    P = M.unflatten(rounded_theta(theta, K), K)
    h1 = M.bf16_round(np.maximum(X @ P["W1"].T + P["b1"], 0))
    h2 = M.bf16_round(np.maximum(h1 @ P["W2"].T + P["b2"], 0))
    return 0.5 * (np.tanh(h2 @ P["w3"] + P["b3"][0]) + 1)


def positions(game, rows, cols, n, seed):
    s = G.reset(game, rows, cols, n)
    G.rollout_from(s, seed=seed, stop_ply=W.ply_samples(n, 3, rows * cols // 2, seed))
    return s


@pytest.mark.parametrize("name,game,rows,cols", [("othello", G.OTHELLO, 8, 8), ("hex11", G.HEX, 11, 11),
                                                 ("c4", G.C4, 6, 7)])
def test_pack_inputs_matches_encoding(L, name, game, rows, cols):
    n = 300
    s = positions(game, rows, cols, n, 1)
    env = L.Env(game, rows, cols, n)
    env.set_state(*(torch.from_numpy(x) for x in (s.board, s.to_move, s.ply, s.passes, s.outcome)))
    K = W.net_in_pad(rows * cols)
    x = torch.empty(n, K, dtype=torch.int16, device="cuda")
    L.ludax_pack_inputs(env.handle, x, K)
    got = x.view(torch.bfloat16).float().cpu().numpy()
    assert (got == M.encode(s.board, s.to_move, K)).all()


@pytest.mark.parametrize("cells,B", [(64, 256), (121, 384), (64, 1280)])
def test_forward_matches_oracle(L, cells, B):
    K = W.net_in_pad(cells)
    theta = W.init_params(cells, 7)
    theta[M.num_params(K) - 1] = 0.1                      # nonzero output bias
    rng = np.random.default_rng(cells)
    X = np.zeros((B, K))
    X[:, :2 * cells + 1] = rng.random((B, 2 * cells + 1)) < 0.3
    net = L.Net(cells, 2048)
    assert (net.in_pad, net.hidden, net.num_params) == (K, 512, M.num_params(K))
    net.set_params(torch.from_numpy(theta).cuda())
    ref = forward_bf16(theta, X, K)
    exact, _ = M.forward(theta.astype(np.float64), X, K)
    for path in (1, 2, 0):  # one-launch tcgen05 MLP, tcgen05 layer by layer, mma.sync
        net.set_tensor_path(path)
        p = net.forward(bf16_bits(X)).cpu().numpy()
        assert np.abs(p - ref).max() < 5e-4
        assert np.abs(p - exact).max() < 2e-2
    assert L.ludax_device_error() == 0
    assert np.allclose(net.get_params().cpu().numpy(), theta)


def grad_bf16(theta, X, y, K, with_bounds=False):
    """fp64 gradient with the kernels' rounding points: BF16 weights, BF16
    hidden activations, and the hidden-layer gradients dZ2 and dZ1 rounded to
    BF16 before the contractions that read them (db2 sums dZ2 unrounded).
    With with_bounds, also each parameter block's element-wise error scales
    (S, m): every gradient element is a sum over the batch of products a_b c_b
    of a row factor and a column factor; S = sum_b |a_b| |c_b| and m =
    max_b |a_b| * max_b |c_b| (a bound on the largest single term)."""
    P = M.unflatten(rounded_theta(theta, K), K)
    B = X.shape[0]
    h1 = M.bf16_round(np.maximum(X @ P["W1"].T + P["b1"], 0))
    h2 = M.bf16_round(np.maximum(h1 @ P["W2"].T + P["b2"], 0))
    v = np.tanh(h2 @ P["w3"] + P["b3"][0])
    g3 = 2.0 * (0.5 * (v + 1) - y) / B * 0.5 * (1 - v * v)
    dz2 = np.outer(g3, P["w3"]) * (h2 > 0)
    dz2b = M.bf16_round(dz2)
    dz1 = M.bf16_round((dz2b @ P["W2"]) * (h1 > 0))
    g = {"W1": dz1.T @ X, "b1": dz1.sum(0), "W2": dz2b.T @ h1, "b2": dz2.sum(0), "w3": h2.T @ g3,
         "b3": np.array([g3.sum()])}
    if not with_bounds:
        return M.flatten(g, K)
    one = np.ones((B, 1))
    factors = {"W1": (dz1, X), "b1": (dz1, one), "W2": (dz2b, h1), "b2": (dz2, one), "w3": (g3[:, None], h2),
               "b3": (g3[:, None], one)}
    bounds = {}
    for name, (a, c) in factors.items():
        a, c = np.abs(a), np.abs(c)
        S = a.T @ c
        m = np.outer(a.max(0), c.max(0))
        if name == "w3":  # w3's element j is sum_b g3_b h2[b, j]: a column vector, like g["w3"]
            S, m = S.ravel(), m.ravel()
        bounds[name] = (S.reshape(g[name].shape), m.reshape(g[name].shape))
    return M.flatten(g, K), bounds


def blocks_close(g, want, K, rel_tol, cos_tol):
    G_, Wt = M.unflatten(g, K), M.unflatten(want, K)
    for name, _ in M.param_shapes(K):
        a, b = G_[name].ravel(), Wt[name].ravel()
        rel = np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-12)
        cos = a @ b / max(np.linalg.norm(a) * np.linalg.norm(b), 1e-30)
        assert rel < rel_tol and cos > cos_tol, (name, rel, cos)


U_BF16, U_FP32 = 2.0 ** -8, 2.0 ** -24


def elements_close(g, want, bounds, K, B):
    """Every element of every block: |g - ref| <= 2^-8 |ref| + 8 sqrt(B) 2^-24 S + 2^-5 m.

    The three terms: (1) one BF16 rounding of the result's dominant factor,
    relative to the element; (2) FP32 accumulation of the B products in any
    order and split, at the probabilistic rate sqrt(B) u (Higham and Mary,
    2019) with a factor 8 of margin, relative to the sum of the products'
    magnitudes S; (3) a BF16 intermediate (hidden activation, dZ2, dZ1) that
    the kernel rounds to the neighbouring BF16 value because its FP32 input
    sat next to a rounding boundary: each such factor moves its term by at
    most 2^-8 of it (2^-7 for the two factors of a term), and up to four such
    terms per element are allowed, each bounded by m.  A wrong sign costs
    2 |ref| and a dropped row one whole term, far above the bound."""
    G_, Wt = M.unflatten(g, K), M.unflatten(want, K)
    worst = {}
    for name, _ in M.param_shapes(K):
        S, m = bounds[name]
        err = np.abs(G_[name] - Wt[name])
        tol = U_BF16 * np.abs(Wt[name]) + 8 * np.sqrt(B) * U_FP32 * S + 4 * 2 * U_BF16 * m
        # where every product is zero (padded columns, units that never fire) the bound is 0: exact zeros
        ratio = np.where(tol > 0, err / np.where(tol > 0, tol, 1.0), np.where(err > 0, np.inf, 0.0))
        k = np.unravel_index(np.argmax(ratio), ratio.shape)
        worst[name] = float(ratio[k])
        assert ratio[k] <= 1.0, (name, k, float(G_[name][k]), float(Wt[name][k]), float(tol[k]))
    return worst


def check_gradient(g, theta, X, y, K, cells, loss=None):
    """g (flat, from the kernels): element by element within the bound of
    elements_close of the fp64 gradient taken with the kernels' BF16 rounding
    points; per parameter block within 2e-3 of it in relative L2 norm; and
    within the BF16 rounding error (a few percent at small batches, where few
    rows average it out) of the plain fp64 gradient of the same BF16 weights."""
    th = rounded_theta(theta, K)
    if loss is not None:
        assert abs(loss - M.loss(th, X, y, K)) < 1e-3 * max(1.0, M.loss(th, X, y, K))
    want, bounds = grad_bf16(theta, X, y, K, with_bounds=True)
    elements_close(g, want, bounds, K, X.shape[0])
    blocks_close(g, want, K, 2e-3, 0.99999)
    blocks_close(g, M.grad(th, X, y, K), K, 6e-2, 0.998)
    # padded input columns never receive gradient
    assert np.abs(M.unflatten(g, K)["W1"][:, 2 * cells + 1:]).max() == 0.0


# B = 128: two K blocks, so two splits of the weight gradients; B = 4736 =
# 37 x 128: 74 K blocks over 18 (dW2) and 37 (dW1) splits, unequal in size;
# 42 cells: 85 inputs padded to 128 columns, so dW1 (N = 128, not a multiple
# of the 256-column tile) stays on mma.sync while the rest runs on tcgen05.
@pytest.mark.parametrize("cells,B", [(64, 512), (121, 256), (64, 128), (64, 4736), (42, 384)])
# tensor path 1: both forward layers in one launch; 2: one launch per layer; 0: mma.sync throughout
@pytest.mark.parametrize("path", [1, 2, 0])
def test_gradient_matches_oracle(L, cells, B, path):
    K = W.net_in_pad(cells)
    theta = W.init_params(cells, 3)
    rng = np.random.default_rng(5)
    X = np.zeros((B, K))
    X[:, :2 * cells + 1] = rng.random((B, 2 * cells + 1)) < 0.3
    y = rng.random(B)
    net = L.Net(cells, max(1024, B))
    net.set_params(torch.from_numpy(theta).cuda())
    net.set_tensor_path(path)
    g, loss = net.grad(bf16_bits(X), torch.from_numpy(y.astype(np.float32)).cuda())
    assert L.ludax_device_error() == 0
    check_gradient(g.cpu().numpy().astype(np.float64), theta, X, y, K, cells, loss.item())


def test_gradient_training_batch(L):
    """The training batch (65,536 rows of Othello inputs): the tcgen05
    forward and backward (one-launch and per-layer forward) against the fp64
    oracle, and against the mma.sync path."""
    cells, B = 64, 65536
    K = W.net_in_pad(cells)
    theta = W.init_params(cells, 9)
    rng = np.random.default_rng(8)
    X = np.zeros((B, K))
    X[:, :2 * cells + 1] = rng.random((B, 2 * cells + 1)) < 0.3
    y = rng.random(B)
    net = L.Net(cells, B)
    net.set_params(torch.from_numpy(theta).cuda())
    xb, yb = bf16_bits(X), torch.from_numpy(y.astype(np.float32)).cuda()
    grads = {}
    for path in (1, 2, 0):
        net.set_tensor_path(path)
        g, _ = net.grad(xb, yb)
        grads[path] = g.cpu().numpy().astype(np.float64)
    assert L.ludax_device_error() == 0
    check_gradient(grads[1], theta, X, y, K, cells)
    check_gradient(grads[2], theta, X, y, K, cells)
    a, b = grads[1], grads[0]
    assert np.linalg.norm(a - b) / np.linalg.norm(b) < 1e-2


@pytest.mark.parametrize("path", [1, 2, 0])
def test_training_is_deterministic(L, path):
    """Every partial sum of the backward pass (split-K weight gradients, row
    sums of the biases, the loss) is reduced in a fixed order, so the same
    batch gives the same gradient, and the same Adam step the same
    parameters, bit for bit (4,736 rows: unequal splits, a ragged last chunk)."""
    cells, B = 64, 4736
    K = W.net_in_pad(cells)
    rng = np.random.default_rng(21)
    X = np.zeros((B, K))
    X[:, :2 * cells + 1] = rng.random((B, 2 * cells + 1)) < 0.3
    xb, yb = bf16_bits(X), torch.from_numpy(rng.random(B).astype(np.float32)).cuda()
    theta = torch.from_numpy(W.init_params(cells, 4)).cuda()
    net = L.Net(cells, B)
    net.set_tensor_path(path)
    net.set_params(theta)
    g1, l1 = net.grad(xb, yb)
    g2, l2 = net.grad(xb, yb)
    assert torch.equal(g1, g2) and torch.equal(l1, l2)
    runs = []
    for _ in range(2):
        net.set_params(theta)  # also resets Adam's moments and step count
        losses = [net.train_step(xb, yb, 1e-3).clone() for _ in range(3)]
        runs.append((net.get_params().clone(), torch.cat(losses)))
    assert torch.equal(runs[0][0], runs[1][0]) and torch.equal(runs[0][1], runs[1][1])
    assert L.ludax_device_error() == 0
    net.close()


def test_checkpoint_resumes_training_exactly(L, tmp_path):
    """Training interrupted by a checkpoint (parameters, both Adam moments,
    the step count; written to a file and read back into a fresh net) goes on
    exactly as if uninterrupted, and the restored net predicts the same."""
    from paper_2506_22609_b300 import valuenet as V

    cells, B = 64, 1024
    K = W.net_in_pad(cells)
    rng = np.random.default_rng(31)
    X = np.zeros((B, K))
    X[:, :2 * cells + 1] = rng.random((B, 2 * cells + 1)) < 0.3
    xb, yb = bf16_bits(X), torch.from_numpy(rng.random(B).astype(np.float32)).cuda()
    theta = torch.from_numpy(W.init_params(cells, 6)).cuda()
    a = L.Net(cells, B)
    a.set_params(theta)
    for _ in range(3):
        a.train_step(xb, yb, 1e-3)
    path = str(tmp_path / "net.ckpt")
    V.save_checkpoint(a, path)
    for _ in range(4):
        a.train_step(xb, yb, 1e-3)
    b = L.Net(cells, B)
    assert V.load_checkpoint(b, path) == 3
    for _ in range(4):
        b.train_step(xb, yb, 1e-3)
    pa, ma, va, ta = a.get_state()
    pb, mb, vb, tb = b.get_state()
    assert ta == tb == 7
    assert torch.equal(pa, pb) and torch.equal(ma, mb) and torch.equal(va, vb)
    assert torch.equal(a.forward(xb), b.forward(xb))
    c = L.Net(121, B)  # a net of another shape refuses it
    with pytest.raises(ValueError):
        V.load_checkpoint(c, path)
    for n in (a, b, c):
        n.close()


def test_adam_step_matches_oracle(L):
    cells, B = 64, 256
    K = W.net_in_pad(cells)
    theta = W.init_params(cells, 11)
    rng = np.random.default_rng(2)
    X = np.zeros((B, K))
    X[:, :129] = rng.random((B, 129)) < 0.3
    y = rng.random(B)
    net = L.Net(cells, 256)
    net.set_params(torch.from_numpy(theta).cuda())
    xb, yb = bf16_bits(X), torch.from_numpy(y.astype(np.float32)).cuda()
    th, m, v = theta.astype(np.float64), np.zeros(theta.size), np.zeros(theta.size)
    for t in (1, 2, 3):
        g, _ = net.grad(xb, yb)
        net.train_step(xb, yb, 1e-3)
        th, m, v = M.adam_step(th, m, v, g.cpu().numpy().astype(np.float64), t, 1e-3)
        got = net.get_params().cpu().numpy()
        assert np.abs(got - th).max() < 2e-6, t
        th = got.astype(np.float64)  # follow the fp32 trajectory


def test_training_fits_a_fixed_target(L):
    # A learnable target: the label is the fraction of P1 stones among the
    # first 16 cells, so the loss must fall well below the label variance.
    cells, B = 64, 2048
    K = W.net_in_pad(cells)
    rng = np.random.default_rng(0)
    X = np.zeros((B, K))
    X[:, :129] = rng.random((B, 129)) < 0.5
    y = X[:, :16].mean(1)
    net = L.Net(cells, B)
    net.set_params(torch.from_numpy(W.init_params(cells, 1)).cuda())
    xb, yb = bf16_bits(X), torch.from_numpy(y.astype(np.float32)).cuda()
    first = net.train_step(xb, yb, 1e-3).item()
    for _ in range(300):
        last = net.train_step(xb, yb, 1e-3).item()
    assert last < 0.1 * first and last < 0.1 * y.var()


# K = 1, 2: the mean forms p from the head partials itself; K = 4: through the
# head's finish; 200 positions leave padding rows up to 256 (zeroed by the leaf kernel)
@pytest.mark.parametrize("Kc", [1, 2, 4])
@pytest.mark.parametrize("name,game,rows,cols", [("othello", G.OTHELLO, 8, 8), ("hex7", G.HEX, 7, 7)])
def test_truncated_value_matches_oracle(L, name, game, rows, cols, Kc):
    n, plies, seed = 200, 8, 99
    cells = rows * cols
    K = W.net_in_pad(cells)
    s = positions(game, rows, cols, n, 4)
    env = L.Env(game, rows, cols, n, env_offset=10)
    env.set_state(*(torch.from_numpy(x) for x in (s.board, s.to_move, s.ply, s.passes, s.outcome)))
    theta = W.init_params(cells, 8)
    net = L.Net(cells, 1024)
    net.set_params(torch.from_numpy(theta).cuda())
    val = torch.empty(n, dtype=torch.float32, device="cuda")
    L.ludax_truncated_value(env.handle, net.handle, seed, Kc, plies, val)
    val = val.cpu().numpy()
    want = np.zeros(n)
    for j in range(Kc):
        t = s.copy()
        G.rollout_from(t, seed=seed + j, env_offset=10, stop_ply=(t.ply + plies).astype(np.int16))
        p = forward_bf16(theta, M.encode(t.board, t.to_move, K), K)
        res = np.where(t.outcome == 1, 1.0, np.where(t.outcome == 2, 0.0, 0.5))
        want += np.where(t.outcome >= 0, res, p)
    want /= Kc
    assert np.abs(val - want).max() < 5e-4


def subset(s, idx):
    """The positions idx of a States batch, as a new batch."""
    t = G.States(s.game, s.rows, s.cols, len(idx))
    for k in ("board", "to_move", "ply", "passes", "outcome"):
        setattr(t, k, np.ascontiguousarray(getattr(s, k)[idx]))
    return t


@pytest.mark.parametrize("cells", [64, 121])
def test_forward_large_batch_sampled(L, cells):
    """Inference at a batch where every CTA of the persistent launch runs
    several 128-row blocks (595 blocks over at most 148 SMs, a ragged last
    round): sampled rows from every part of the batch against the oracle."""
    B = 595 * 128
    K = W.net_in_pad(cells)
    theta = W.init_params(cells, 11)
    theta[M.num_params(K) - 1] = -0.05
    rng = np.random.default_rng(cells + 1)
    X = np.zeros((B, K), np.float32)
    X[:, :2 * cells + 1] = rng.random((B, 2 * cells + 1)) < 0.3
    net = L.Net(cells, B)
    net.set_params(torch.from_numpy(theta).cuda())
    idx = np.unique(np.concatenate([np.arange(0, B, 211), np.arange(B - 128, B), np.arange(148 * 128, 150 * 128)]))
    ref = forward_bf16(theta, X[idx].astype(np.float64), K)
    xb = bf16_bits(X)
    for path in (1, 2):  # one launch with layer 1 through L2; two layer launches
        net.set_tensor_path(path)
        p = net.forward(xb).cpu().numpy()
        assert L.ludax_device_error() == 0
        assert np.abs(p[idx] - ref).max() < 5e-4
        assert np.isfinite(p).all() and (p > 0).all() and (p < 1).all()


# 24,000 x 4 rows; and the value benchmark's own configurations: 100,000
# positions with K = 8 (Othello, 800,000 rows in one launch of the fused MLP)
# and K = 1 (Hex 11)
@pytest.mark.parametrize("game,rows,cols,n,Kc", [(G.OTHELLO, 8, 8, 24000, 4), (G.OTHELLO, 8, 8, 100000, 8),
                                                 (G.HEX, 11, 11, 100000, 1)], ids=["othello_24k_k4", "othello_100k_k8",
                                                                                  "hex11_100k_k1"])
def test_truncated_value_large_batch_sampled(L, game, rows, cols, n, Kc):
    """The truncated estimator with K * n rows spanning many blocks per CTA
    (only the input columns the first layer needs are read): sampled
    positions against the oracle, each replayed with its own env index."""
    plies, seed = 8, 123
    cells = rows * cols
    K = W.net_in_pad(cells)
    s = positions(game, rows, cols, n, 6)
    env = L.Env(game, rows, cols, n, env_offset=3)
    env.set_state(*(torch.from_numpy(x) for x in (s.board, s.to_move, s.ply, s.passes, s.outcome)))
    theta = W.init_params(cells, 12)
    net = L.Net(cells, (n * Kc + 127) // 128 * 128)  # row capacity: a multiple of 128
    net.set_params(torch.from_numpy(theta).cuda())
    val = torch.empty(n, dtype=torch.float32, device="cuda")
    L.ludax_truncated_value(env.handle, net.handle, seed, Kc, plies, val)
    val = val.cpu().numpy()
    assert L.ludax_device_error() == 0
    idx = np.unique(np.concatenate([np.arange(0, n, 397), np.arange(n - 8, n)]))
    want = np.zeros(len(idx))
    for j in range(Kc):
        for r, e in enumerate(idx):
            t = subset(s, [e])
            G.rollout_from(t, seed=seed + j, env_offset=3 + int(e), stop_ply=(t.ply + plies).astype(np.int16))
            if t.outcome[0] >= 0:
                want[r] += 1.0 if t.outcome[0] == 1 else (0.0 if t.outcome[0] == 2 else 0.5)
            else:
                want[r] += forward_bf16(theta, M.encode(t.board, t.to_move, K), K)[0]
    want /= Kc
    assert np.abs(val[idx] - want).max() < 5e-4
