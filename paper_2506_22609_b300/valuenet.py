"""Learned value estimates: data, training and evaluation of the value net.

    python -m paper_2506_22609_b300.valuenet --game othello [--n-train 2000000] [--epochs 100]

Pipeline (every compute step is a libludax kernel; this module only moves
handles, sizes and seeds around):
  1. positions: uniform-random playouts from the start position stopped at a
     ply t drawn uniformly from 10..40 (ludax_rollout with stop plies); a
     playout that ends before t is rejected and replaced by a fresh one;
  2. labels: the fraction of 64 uniform-random playouts from the position
     that P1 wins, draws counting one half (ludax_rollout_value);
  3. training: batches of 65,536 positions, Adam at lr 1e-3
     (ludax_net_train_step), the batch order shuffled each epoch, for up to
     max_epochs epochs; the epoch kept is the one whose net is closest (mean
     absolute error) to a 256-playout reference of the VALIDATION positions;
  4. selection on the validation positions, never on the held-out ones: the
     smallest number K of truncated continuations (8 random plies, then the
     net: ludax_truncated_value) and the smallest number M of full playouts
     (ludax_rollout_value) whose mean absolute error against the validation
     reference is at most the target;
  5. evaluation, once, on held-out positions against their own 256-playout
     reference: every K and M (mean absolute error and estimates per second),
     the selected K and M, and the comparison at an equal time budget (the
     full-playout estimator with the largest M that fits in the selected
     truncated estimator's time).
Checkpoints (save_checkpoint / load_checkpoint) hold the parameters, both
Adam moments and the step count, so training resumes bit for bit.
"""
from __future__ import annotations

import argparse
import json
import os
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


def train(net, x, y, batch, epochs, lr, seed, x_val=None, y_val=None, log=None, keep_best=False):
    """Adam over shuffled batches; with x_val, each epoch's validation MAE
    is recorded, and with keep_best the parameters of the epoch with the
    smallest one are restored at the end.  Returns (history, seconds of
    training steps, steps, the epoch kept)."""
    n = x.shape[0]
    nb = n // batch
    rng = np.random.default_rng(seed)
    hist = []
    t_train = 0.0
    steps = 0
    best, best_ep, best_params = float("inf"), epochs, None
    for ep in range(epochs):
        losses = []
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for b in rng.permutation(nb):
            loss = net.train_step(x[b * batch:(b + 1) * batch], y[b * batch:(b + 1) * batch], lr)
            losses.append(loss)
            steps += 1
        torch.cuda.synchronize()
        t_train += time.perf_counter() - t0
        rec = {"epoch": ep + 1, "train_loss": float(torch.stack(losses).mean().item())}
        if x_val is not None:
            p = predict(net, x_val)
            rec["val_mae"] = float((p - y_val).abs().mean().item())
            if keep_best and rec["val_mae"] < best:
                best, best_ep, best_params = rec["val_mae"], ep + 1, net.get_params()
        hist.append(rec)
        if log:
            log(rec)
    if keep_best and best_params is not None:
        net.set_params(best_params)
    torch.cuda.synchronize()
    return hist, t_train, steps, best_ep


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


def estimator_table(env, net, ref, seed, Ms, Ks, plies, timed=True):
    """MAE against ref (and estimates/s) of full playouts for every M and of
    the truncated estimator for every K on the positions of env."""
    n = env.num_envs
    full, trunc = [], []
    for M in Ms:
        fn = lambda: env.rollout_value(seed + 100000 * M, M)  # noqa: E731
        v, dt = cuda_time_median(fn) if timed else (fn(), None)
        full.append({"M": M, "mae": float((v - ref).abs().mean().item()),
                     "estimates_per_s": n / dt if dt else None, "seconds": dt})
    for K in Ks:
        val = torch.empty(n, dtype=torch.float32, device="cuda")
        fn = lambda: L.ludax_truncated_value(env.handle, net.handle, seed + 7777 + 1000 * K, K, plies, val)  # noqa: E731
        _, dt = cuda_time_median(fn) if timed else (fn(), None)
        trunc.append({"K": K, "plies": plies, "mae": float((val - ref).abs().mean().item()),
                      "estimates_per_s": n / dt if dt else None, "seconds": dt})
    return full, trunc


def first_at(rows, target):
    ok = [x for x in rows if x["mae"] <= target]
    return ok[0] if ok else rows[-1]


def evaluate(env, net, ref, seed, Ms=(1, 2, 4, 8, 16, 32, 64, 128), Ks=(1, 2, 4, 8, 16), plies=8, target=0.05,
             K_sel=None, M_sel=None, M_eq=None):
    """The held-out evaluation: every estimator's MAE against the reference
    and its speed; K_sel / M_sel are the counts chosen on the validation
    positions for the target, M_eq the full-playout count that matched the
    selected truncated estimator's validation MAE (this function never
    chooses a count from its own errors)."""
    n = env.num_envs
    net, owned = inference_net(net, n * max(Ks))
    full, trunc = estimator_table(env, net, ref, seed, Ms, Ks, plies)
    res = {"full_playouts": full, "truncated": trunc}
    pnet = predict(net, pack(env, net.in_pad))
    res["net_only_mae"] = float((pnet - ref).abs().mean().item())
    res["inference_rows"] = net.max_batch
    if owned:
        net.close()
    # noise of the reference itself: sd of a 256-sample mean, as an expected absolute value
    r = ref.double()
    res["reference_noise_mae"] = float((torch.sqrt(r * (1 - r) / 256) * (2 / np.pi) ** 0.5).mean().item())
    res["target_mae"] = target
    if K_sel is not None:
        t = next(x for x in trunc if x["K"] == K_sel)
        f = next(x for x in full if x["M"] == M_sel)
        res["truncated_selected"], res["full_selected"] = t, f
        res["gain_estimates_per_s"] = t["estimates_per_s"] / f["estimates_per_s"]
        if M_eq is not None:
            fe = next(x for x in full if x["M"] == M_eq)
            res["equal_mae"] = {"truncated_K": K_sel, "truncated_mae": t["mae"],
                                "truncated_estimates_per_s": t["estimates_per_s"], "full_M": M_eq,
                                "full_mae": fe["mae"], "full_estimates_per_s": fe["estimates_per_s"],
                                "gain": t["estimates_per_s"] / fe["estimates_per_s"]}
        # equal time budget: the most full playouts per position that fit in the truncated estimator's time
        fit = [x for x in full if x["seconds"] <= t["seconds"]]
        res["equal_time"] = {"truncated_K": K_sel, "truncated_mae": t["mae"], "seconds": t["seconds"],
                             "full_M": fit[-1]["M"] if fit else 0,
                             "full_mae": fit[-1]["mae"] if fit else float((0.5 - ref).abs().mean().item())}
    return res


def run(game="othello", n_train=2_000_000, n_val=65_536, n_eval=100_000, batch=65_536, epochs=100, lr=1e-3,
        label_R=64, ref_R=256, seed=5, target=0.05, Ks=(1, 2, 4, 8, 16), Ms=(1, 2, 4, 8, 16, 32, 64, 128),
        log=None):
    g, rows, cols = GAMES[game]
    cells = rows * cols
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    env_tr, off = sample_positions(g, rows, cols, n_train, seed, 0)
    env_va, off = sample_positions(g, rows, cols, n_val, seed + 1, off)
    env_ev, off = sample_positions(g, rows, cols, n_eval, seed + 2, off)
    y_tr, t_lab = cuda_time(lambda: env_tr.rollout_value(seed * 7919 + 1, label_R))
    ref_va = env_va.rollout_value(seed * 7919 + 2, ref_R)
    ref = env_ev.rollout_value(seed * 7919 + 3, ref_R)
    in_pad = W.net_in_pad(cells)
    x_tr, x_va = pack(env_tr, in_pad), pack(env_va, in_pad)
    torch.cuda.synchronize()
    t_data = time.perf_counter() - t0
    net = L.Net(cells, batch)
    net.set_params(torch.from_numpy(W.init_params(cells, seed)).cuda())
    untrained_val_mae = float((predict(net, x_va) - ref_va).abs().mean().item())
    hist, t_train, steps, kept = train(net, x_tr, y_tr, batch, epochs, lr, seed, x_va, ref_va, log, keep_best=True)
    # K and M chosen on the validation positions against their own reference
    vnet, owned = inference_net(net, n_val * max(Ks))
    vfull, vtrunc = estimator_table(env_va, vnet, ref_va, seed * 31 + 5, Ms, Ks, 8, timed=False)
    if owned:
        vnet.close()
    t_sel = first_at(vtrunc, target)
    K_sel, M_sel = t_sel["K"], first_at(vfull, target)["M"]
    M_eq = first_at(vfull, t_sel["mae"])["M"]  # full playouts as accurate as the selected truncated estimator
    ev = evaluate(env_ev, net, ref, seed * 31 + 17, Ms=Ms, Ks=Ks, target=target, K_sel=K_sel, M_sel=M_sel,
                  M_eq=M_eq)
    out = {"game": game, "n_train": n_train, "n_val": n_val, "n_eval": n_eval, "batch": batch, "epochs": epochs,
           "epoch_kept": kept, "lr": lr, "label_playouts": label_R, "reference_playouts": ref_R,
           "data_seconds": t_data, "label_playouts_per_s": n_train * label_R / t_lab, "train_seconds": t_train,
           "train_steps": steps, "untrained_val_mae": untrained_val_mae, "history": hist,
           "validation": {"truncated": vtrunc, "full_playouts": vfull, "K": K_sel, "M": M_sel, "M_equal_mae": M_eq},
           "eval": ev}
    for e in (env_tr, env_va, env_ev):
        e.close()
    net.close()
    return out


# --------------------------------------------------------------- checkpoints --
# One little-endian file: the 8-byte magic b"LUDAXNET", six int64 -- format
# version, cells, input width, hidden width, number of parameters, Adam steps
# taken -- then the FP32 parameters and Adam's first and second moments,
# num_params each.  Restoring it continues training exactly where it stood
# (ludax_net_set_state).
CKPT_MAGIC, CKPT_VERSION = b"LUDAXNET", 1


def write_checkpoint(path, cells, in_pad, hidden, steps, params, m, v):
    """Writes the arrays (float32, num_params each) under the header; the
    file appears whole or not at all (written aside, then renamed)."""
    arrays = [np.ascontiguousarray(a, dtype="<f4") for a in (params, m, v)]
    n = arrays[0].size
    if any(a.size != n for a in arrays):
        raise ValueError("parameters and moments differ in length")
    head = np.array([CKPT_VERSION, cells, in_pad, hidden, n, steps], dtype="<i8")
    tmp = f"{path}.tmp"
    with open(tmp, "wb") as f:
        f.write(CKPT_MAGIC)
        f.write(head.tobytes())
        for a in arrays:
            f.write(a.tobytes())
    os.replace(tmp, path)


def read_checkpoint(path):
    """The header fields and the three arrays; ValueError if the file is not
    a checkpoint of this format or is cut short."""
    with open(path, "rb") as f:
        data = f.read()
    if data[:8] != CKPT_MAGIC or len(data) < 56:
        raise ValueError(f"{path}: not a value-net checkpoint")
    version, cells, in_pad, hidden, n, steps = (int(x) for x in np.frombuffer(data, "<i8", 6, 8))
    if version != CKPT_VERSION:
        raise ValueError(f"{path}: checkpoint format {version}, expected {CKPT_VERSION}")
    if n < 1 or len(data) != 56 + 12 * n:
        raise ValueError(f"{path}: {len(data)} bytes, expected {56 + 12 * n}")
    arr = np.frombuffer(data, "<f4", 3 * n, 56).reshape(3, n)
    return {"cells": cells, "in_pad": in_pad, "hidden": hidden, "steps": steps,
            "params": arr[0].copy(), "m": arr[1].copy(), "v": arr[2].copy()}


def save_checkpoint(net, path):
    p, m, v, steps = net.get_state()
    torch.cuda.synchronize()
    write_checkpoint(path, net.cells, net.in_pad, net.hidden, steps, p.cpu().numpy(), m.cpu().numpy(),
                     v.cpu().numpy())


def load_checkpoint(net, path):
    """Restores a checkpoint into a net of the same shape; returns the Adam steps it had taken."""
    c = read_checkpoint(path)
    if (c["cells"], c["in_pad"], c["hidden"], c["params"].size) != (net.cells, net.in_pad, net.hidden,
                                                                      net.num_params):
        raise ValueError(f"{path}: a net of {c['cells']} cells, {c['in_pad']} inputs, {c['hidden']} hidden units")
    net.set_state(*(torch.from_numpy(c[k]) for k in ("params", "m", "v")), c["steps"])
    return c["steps"]


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--game", default="othello", choices=sorted(GAMES))
    ap.add_argument("--n-train", type=int, default=2_000_000)
    ap.add_argument("--n-eval", type=int, default=100_000)
    ap.add_argument("--epochs", type=int, default=100)
    ap.add_argument("--seed", type=int, default=5)
    a = ap.parse_args()
    res = run(a.game, n_train=a.n_train, n_eval=a.n_eval, epochs=a.epochs, seed=a.seed,
              log=lambda r: print(json.dumps(r), flush=True))
    print(json.dumps(res))


if __name__ == "__main__":
    main()
