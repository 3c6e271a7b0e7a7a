"""Learned value estimates: data, training and evaluation of the value net.

    python -m paper_2506_22609_b300.valuenet --game othello [--n-train 2000000] [--epochs 30]

Pipeline (every compute step is a libludax kernel; this module only moves
handles, sizes and seeds around):
  1. positions: uniform-random playouts from the start position stopped at a
     ply t drawn uniformly from 10..40 (ludax_rollout with stop plies); a
     playout that ends before t is rejected and replaced by a fresh one;
  2. labels: the fraction of 64 uniform-random playouts from the position
     that P1 wins, draws counting one half (ludax_rollout_value);
  3. training: batches of 65,536 positions, Adam at lr 1e-3
     (ludax_net_train_step), the batch order shuffled each epoch;
  4. evaluation on held-out positions against a 256-playout reference
     estimate: the truncated estimator (K continuations of 8 random plies,
     then the net: ludax_truncated_value) and the full-playout estimator with
     M playouts (ludax_rollout_value), each as mean absolute error and
     estimates per second.
"""
from __future__ import annotations

import argparse
import json
import time

import numpy as np
import torch

from . import ludax as L
from . import workloads as W

GAMES = {"othello": (L.LUDAX_GAME_OTHELLO, 8, 8), "hex11": (L.LUDAX_GAME_HEX, 11, 11)}


def sample_positions(game, rows, cols, n, seed, env_offset=0, lo=10, hi=40):
    """An Env holding n positions, each the state of a random playout at a
    ply drawn from lo..hi; returns (env, next unused env offset)."""
    cells = rows * cols
    keep_board, keep_tm, keep_ply, keep_ps = [], [], [], []
    have, off, rnd = 0, env_offset, 0
    while have < n:
        m = int((n - have) * 1.02) + 1024
        env = L.Env(game, rows, cols, m, env_offset=off)
        stop = torch.from_numpy(W.ply_samples(m, lo, hi, seed * 1000003 + rnd)).cuda()
        out, _ = env.rollout(seed, from_start=True, write_back=True, stop_ply=stop)
        b, tm, ply, ps, oc = (t.cpu().numpy() for t in env.get_state())
        ok = np.flatnonzero(oc == -1)[: n - have]
        keep_board.append(b[ok]); keep_tm.append(tm[ok]); keep_ply.append(ply[ok]); keep_ps.append(ps[ok])
        have += ok.size
        off += m
        rnd += 1
        env.close()
    env = L.Env(game, rows, cols, n)
    board = np.concatenate(keep_board).reshape(n, cells)
    env.set_state(torch.from_numpy(board), torch.from_numpy(np.concatenate(keep_tm)),
                  torch.from_numpy(np.concatenate(keep_ply)), torch.from_numpy(np.concatenate(keep_ps)),
                  torch.full((n,), -1, dtype=torch.int8))
    return env, off


def pack(env, in_pad):
    x = torch.empty(env.num_envs, in_pad, dtype=torch.int16, device="cuda")
    L.ludax_pack_inputs(env.handle, x, in_pad)
    return x


def cuda_time(fn):
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    a.record()
    out = fn()
    b.record()
    torch.cuda.synchronize()
    return out, a.elapsed_time(b) / 1e3


def cuda_time_median(fn, warmup=2, reps=5):
    """fn's result and its median time over `reps` timed calls after `warmup`
    untimed ones (the first call of a shape also pays one-time setup)."""
    for _ in range(warmup):
        fn()
    times = []
    for _ in range(reps):
        out, dt = cuda_time(fn)
        times.append(dt)
    return out, float(np.median(times))


def train(net, x, y, batch, epochs, lr, seed, x_val=None, y_val=None, log=None):
    n = x.shape[0]
    nb = n // batch
    rng = np.random.default_rng(seed)
    hist = []
    t0 = time.perf_counter()
    steps = 0
    for ep in range(epochs):
        losses = []
        for b in rng.permutation(nb):
            loss = net.train_step(x[b * batch:(b + 1) * batch], y[b * batch:(b + 1) * batch], lr)
            losses.append(loss)
            steps += 1
        rec = {"epoch": ep + 1, "train_loss": float(torch.stack(losses).mean().item())}
        if x_val is not None:
            p = predict(net, x_val)
            rec["val_mae"] = float((p - y_val).abs().mean().item())
        hist.append(rec)
        if log:
            log(rec)
    torch.cuda.synchronize()
    return hist, time.perf_counter() - t0, steps


def predict(net, x):
    out = []
    for i in range(0, x.shape[0], net.max_batch):
        xb = x[i:i + net.max_batch]
        pad = (-xb.shape[0]) % 128
        if pad:
            xb = torch.cat([xb, torch.zeros(pad, xb.shape[1], dtype=xb.dtype, device=xb.device)])
        out.append(net.forward(xb)[: xb.shape[0] - pad])
    return torch.cat(out)


def inference_net(net, rows):
    """A copy of the trained net whose buffers hold `rows` rows (rounded up to
    128, at most 2^21), so an estimate over all positions is one batch:
    every continuation of every position goes through the dense layers as one
    large GEMM instead of max_batch-sized chunks."""
    rows = min(1 << 21, ((int(rows) + 127) // 128) * 128)
    if rows <= net.max_batch:
        return net, False
    big = L.Net(net.cells, rows)
    big.set_params(net.get_params())
    return big, True


def evaluate(env, net, ref, seed, Ms=(4, 8, 16, 32, 64, 128), Ks=(1, 2, 4, 8, 16), plies=8, target=0.05):
    n = env.num_envs
    res = {"full_playouts": [], "truncated": []}
    net, owned = inference_net(net, n * max(Ks))
    for M in Ms:
        v, dt = cuda_time_median(lambda: env.rollout_value(seed + 100000 * M, M))
        res["full_playouts"].append({"M": M, "mae": float((v - ref).abs().mean().item()),
                                     "estimates_per_s": n / dt, "seconds": dt})
    for K in Ks:
        val = torch.empty(n, dtype=torch.float32, device="cuda")
        _, dt = cuda_time_median(lambda: L.ludax_truncated_value(env.handle, net.handle, seed + 7777 + 1000 * K, K,
                                                                 plies, val))
        res["truncated"].append({"K": K, "plies": plies, "mae": float((val - ref).abs().mean().item()),
                                 "estimates_per_s": n / dt, "seconds": dt})
    pnet = predict(net, pack(env, net.in_pad))
    res["net_only_mae"] = float((pnet - ref).abs().mean().item())
    res["inference_rows"] = net.max_batch
    if owned:
        net.close()
    # noise of the reference itself: sd of a 256-sample mean, as an expected absolute value
    r = ref.double()
    res["reference_noise_mae"] = float((torch.sqrt(r * (1 - r) / 256) * (2 / np.pi) ** 0.5).mean().item())
    ok_m = [x for x in res["full_playouts"] if x["mae"] <= target]
    ok_k = [x for x in res["truncated"] if x["mae"] <= target]
    res["target_mae"] = target
    res["full_at_target"] = ok_m[0] if ok_m else None
    res["truncated_at_target"] = ok_k[0] if ok_k else None
    if ok_m and ok_k:
        res["gain_estimates_per_s"] = ok_k[0]["estimates_per_s"] / ok_m[0]["estimates_per_s"]
    return res


def run(game="othello", n_train=2_000_000, n_val=65_536, n_eval=100_000, batch=65_536, epochs=30, lr=1e-3,
        label_R=64, ref_R=256, seed=5, log=None):
    g, rows, cols = GAMES[game]
    cells = rows * cols
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    env_tr, off = sample_positions(g, rows, cols, n_train, seed, 0)
    env_va, off = sample_positions(g, rows, cols, n_val, seed + 1, off)
    env_ev, off = sample_positions(g, rows, cols, n_eval, seed + 2, off)
    y_tr, t_lab = cuda_time(lambda: env_tr.rollout_value(seed * 7919 + 1, label_R))
    y_va = env_va.rollout_value(seed * 7919 + 2, label_R)
    ref = env_ev.rollout_value(seed * 7919 + 3, ref_R)
    in_pad = W.net_in_pad(cells)
    x_tr, x_va = pack(env_tr, in_pad), pack(env_va, in_pad)
    torch.cuda.synchronize()
    t_data = time.perf_counter() - t0
    net = L.Net(cells, batch)
    net.set_params(torch.from_numpy(W.init_params(cells, seed)).cuda())
    untrained_val_mae = float((predict(net, x_va) - y_va).abs().mean().item())
    hist, t_train, steps = train(net, x_tr, y_tr, batch, epochs, lr, seed, x_va, y_va, log)
    ev = evaluate(env_ev, net, ref, seed * 31 + 17)
    out = {"game": game, "n_train": n_train, "n_val": n_val, "n_eval": n_eval, "batch": batch, "epochs": epochs,
           "lr": lr, "label_playouts": label_R, "reference_playouts": ref_R, "data_seconds": t_data,
           "label_playouts_per_s": n_train * label_R / t_lab, "train_seconds": t_train, "train_steps": steps,
           "untrained_val_mae": untrained_val_mae, "history": hist, "eval": ev}
    for e in (env_tr, env_va, env_ev):
        e.close()
    net.close()
    return out


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--game", default="othello", choices=sorted(GAMES))
    ap.add_argument("--n-train", type=int, default=2_000_000)
    ap.add_argument("--n-eval", type=int, default=100_000)
    ap.add_argument("--epochs", type=int, default=30)
    ap.add_argument("--seed", type=int, default=5)
    a = ap.parse_args()
    res = run(a.game, n_train=a.n_train, n_eval=a.n_eval, epochs=a.epochs, seed=a.seed,
              log=lambda r: print(json.dumps(r), flush=True))
    print(json.dumps(res))


if __name__ == "__main__":
    main()
