"""Benchmark: env steps/s of uniform-random playouts on B300.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                    [--workload c4|ttt|othello|hex11|gomoku|pente|yavalath|line_c5|wolf_sheep|
                                draughts|hasami_shogi|mixed|step_c4]
                    [--no-extras] [--no-cpu-baseline] [--only dense_layer|gavel_library|
                     batch_sweep|value_net|value_estimator|int_peak|train_step|threads_per_env|
                     lanes_per_warp]

One step = one fused playout launch over the whole batch: every env of the
workload is reset to the start position and played to the end of its game
with the counter-based uniform-random policy (legal mask, draw, select,
apply with captures/flips/gravity, terminal and win detection, all in
registers), and each env's outcome and game length are written to HBM.
The default workload is the mixed batch: 1,048,576 envs split evenly over
Tic-Tac-Toe, Connect Four, Reversi and Hex 7x7 / 9x9 / 11x11, seed 3, one
graph-captured launch per step (the largest single-GPU configuration).

Metric: env steps per second = total plies played (passes included) / time.
`value` is device time (CUDA events on the launching stream) with L2 flushed
between steps; `e2e` goes through the C-ABI call with host buffers
(ludax_mixed_plan_launch_host for the mixed batch: descriptors copied from
pinned host memory, the work queue rebuilt on the device, the playouts, and
outcome + game length copied back; ludax_rollout_host for a single game:
start positions in the packed state view in, the same results out).

Under torchrun (N > 1) each rank plays its own disjoint range of global env
ids (weak scaling, no collective on the data path); the step time is the
maximum over ranks.  `--impl reference` times the CPU oracle (plain C, all
host cores) on a bounded sample of the same workload.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "env steps/sec on 1 B300 (random playouts); value estimates/sec at stated MAE"

# Algorithmic 32-bit integer operations per env step of the fused playout,
# counted from the bitboard algorithm with a 3-input logic op counted once:
# RNG draw (13 logic/shift/add + 7 multiply), legal mask, popcount, k-th-bit
# select, apply (Reversi flips), end test.  Reversi's count (437) is within 2%
# of the instructions ncu measures executed per ply (444).
# The parametric line game's count is for its benchmarked instance (9 x 12,
# exactly five, gravity): RNG 20, legal with gravity 18, popcount 5, select 30,
# place 4, four directions x (three doubling shift-ANDs + the two exact-length
# shifts) 248, outcome and turn 9.
ALG_OPS_PER_STEP = {"ttt": 75, "c4": 112, "othello": 437, "hex": 180, "gomoku": 330, "pente": 700,
                    "yavalath": 150, "line": 334}
# Estimates of the same work made before any kernel was written: TTT ~40,
# C4 ~80, Reversi ~350-500 (the count above, 437, lies inside), Hex ~100 + ~40
# per flood round; a random Hex game needs 0.27-0.29 flood rounds per ply on
# 7x7 to 11x11 boards (the incremental edge-set update), so Hex ~112.
PRIOR_OPS_PER_STEP = {"ttt": 40, "c4": 80, "othello": 437, "hex": 112}
# game id of a descriptor (low byte) -> key of the tables above
GAME_KEYS = {0: "ttt", 1: "c4", 2: "othello", 3: "hex", 4: "gomoku", 5: "pente", 6: "yavalath", 7: "line"}

# DRAM bytes per launch of the benchmarked kernel, from the committed ncu
# captures (profiles/); None once the kernel changes until it is captured again.
NCU_TRAFFIC_BYTES = {"mixed6_1048576env_seed3_graph": 4275456}
# thread instructions ncu counts executed per env step (warp instructions x
# active lanes per instruction / plies of the launch), from the same captures
NCU_THREAD_INST_PER_STEP = {"mixed6_1048576env_seed3_graph": round(670130108 * 24.32 / 54553274, 1)}


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=200)
    p.add_argument("--warmup", type=int, default=5)
    p.add_argument("--impl", default="ours", choices=["ours", "reference"])
    p.add_argument("--workload", default="mixed", choices=["c4", "ttt", "othello", "hex11", "gomoku", "pente", "yavalath",
                                                        "line_c5", "wolf_sheep", "draughts", "hasami_shogi", "mixed",
                                                        "step_c4"])
    p.add_argument("--no-extras", action="store_true")
    p.add_argument("--only", choices=["dense_layer", "gavel_library", "batch_sweep", "value_net", "value_estimator",
                                      "int_peak", "train_step", "threads_per_env", "lanes_per_warp"],
                   default=None,
                   help="run one extra measurement alone and print its JSON (a small case for profilers)")
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--no-valuenet", action="store_true", help="skip the value-net (config 5) extra")
    p.add_argument("--cpu-seconds", type=float, default=8.0, help="target wall time of the CPU-baseline sample")
    return p.parse_args()


def workload_cfg(name):
    from paper_2506_22609_b300 import workloads as W

    return {"c4": W.C4_64K, "ttt": W.TTT_1K, "othello": W.OTHELLO_256K, "hex11": W.HEX11_64K, "gomoku": W.GOMOKU_64K,
            "pente": W.PENTE_64K, "yavalath": W.YAVALATH_64K, "line_c5": W.CONNECT5_9X12_64K,
            "wolf_sheep": W.WOLF_SHEEP_64K, "draughts": W.DRAUGHTS_64K, "hasami_shogi": W.HASAMI_64K}[name]


def game_key(cfg):
    return {0: "ttt", 1: "c4", 2: "othello", 3: "hex", 4: "gomoku", 5: "pente", 6: "yavalath", 7: "line",
            8: "wolf_sheep", 9: "draughts", 10: "hasami_shogi"}[cfg.game]


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f), "measured"
    except OSError:
        return {"hbm_gbs": 6400.0, "bf16_tflops": 1800.0, "sm_max_mhz": 2032.0}, "fallback"


# ----------------------------------------------------------------- clocks --
class ClockSampler:
    """Polls NVML's C library (SM clock, max SM clock, clock-event reasons)
    from a thread while the timed region runs."""

    REASONS = {0x4: "sw_power_cap", 0x8: "hw_slowdown", 0x20: "sw_thermal_slowdown",
               0x40: "hw_thermal_slowdown", 0x80: "hw_power_brake_slowdown"}

    def __init__(self, index, period=0.002):
        import ctypes

        self.samples, self.reasons, self.period = [], set(), period
        self.max_mhz, self.err, self.nv = None, "", None
        self._stop = threading.Event()
        try:
            nv = ctypes.CDLL("libnvidia-ml.so.1")
            if nv.nvmlInit_v2() != 0:
                raise RuntimeError("nvmlInit_v2 failed")
            self.h = ctypes.c_void_p()
            # NVML indexes devices by their physical order; map through CUDA_VISIBLE_DEVICES
            vis = os.environ.get("CUDA_VISIBLE_DEVICES")
            phys = int(vis.split(",")[index]) if vis and vis.split(",")[index].isdigit() else index
            if nv.nvmlDeviceGetHandleByIndex_v2(phys, ctypes.byref(self.h)) != 0:
                raise RuntimeError("nvmlDeviceGetHandleByIndex_v2 failed")
            mx = ctypes.c_uint()
            if nv.nvmlDeviceGetMaxClockInfo(self.h, 1, ctypes.byref(mx)) == 0:  # 1 = NVML_CLOCK_SM
                self.max_mhz = mx.value
            self.reason_fn = getattr(nv, "nvmlDeviceGetCurrentClocksEventReasons", None) or \
                nv.nvmlDeviceGetCurrentClocksThrottleReasons
            self.nv, self.ct = nv, ctypes
        except Exception as e:  # no NVML: report no clock record
            self.err = str(e)

    def _run(self):
        c = self.ct.c_uint()
        r = self.ct.c_ulonglong()
        while not self._stop.is_set():
            if self.nv.nvmlDeviceGetClockInfo(self.h, 1, self.ct.byref(c)) == 0:
                self.samples.append(c.value)
            if self.reason_fn(self.h, self.ct.byref(r)) == 0:
                for bit, name in self.REASONS.items():
                    if r.value & bit:
                        self.reasons.add(name)
            time.sleep(self.period)

    def __enter__(self):
        if self.nv:
            self.t = threading.Thread(target=self._run, daemon=True)
            self.t.start()
        return self

    def __exit__(self, *a):
        self._stop.set()
        if self.nv:
            self.t.join()

    def record(self):
        if not self.nv:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "note": "NVML unavailable: " + self.err}
        return {"sm_mhz": statistics.median(self.samples) if self.samples else None, "sm_max_mhz": self.max_mhz,
                "reasons": sorted(self.reasons), "samples": len(self.samples)}


# ------------------------------------------------------------ CPU oracle --
def sample_ranges(cfg, n, desc=None):
    """(offset, count) env ranges of a CPU sample of n envs: the first n envs of
    a single-game batch; for a mixed batch laid out in game blocks, an equal
    share from the start of every block, so every game is in the sample in
    its batch proportion."""
    if desc is None:
        return [(0, n)]
    import numpy as np

    starts = [0] + [int(i) for i in np.nonzero(desc[1:] != desc[:-1])[0] + 1]
    ends = starts[1:] + [len(desc)]
    k = max(1, n // len(starts))
    return [(a, min(k, b - a)) for a, b in zip(starts, ends)]


def cpu_oracle_rate(cfg, seconds, desc=None):
    """The CPU oracle as it stands (plain C, -O2), all host cores via threads
    (ctypes releases the GIL), on a sample of the workload's envs sized to
    take about `seconds`.  Returns (steps/s, cores, sample description)."""
    from concurrent.futures import ThreadPoolExecutor

    import numpy as np

    from oracle import games as OG

    cores = len(os.sched_getaffinity(0))

    def run(off, n):
        if n <= 0:
            return 0
        if desc is not None:
            _, p = OG.rollout_mixed(desc[off:off + n], cfg.seed, env_offset=off)
        else:
            gid = cfg.game if cfg.game != 7 else 7 | (cfg.line << 8) | (cfg.flags << 12)
            _, p, _ = OG.rollout_start(gid, cfg.rows, cfg.cols, n, cfg.seed, env_offset=off)
        return int(p.astype(np.int64).sum())

    total_envs = cfg.num_envs
    # calibrate on one core with a small sample of the same composition
    n0 = 256 if desc is None else 64 * len(sample_ranges(cfg, 64, desc))
    t0 = time.perf_counter()
    for off, k in sample_ranges(cfg, n0, desc):
        run(off, k)
    per_env = max((time.perf_counter() - t0) / n0, 1e-7)
    n = int(min(total_envs, max(cores * 64, seconds * cores / per_env)))
    chunks = []
    for off, k in sample_ranges(cfg, n, desc):
        step = (k + cores - 1) // cores
        chunks += [(off + i, min(step, k - i)) for i in range(0, k, step)]
    t0 = time.perf_counter()
    with ThreadPoolExecutor(cores) as ex:
        steps = sum(ex.map(lambda c: run(*c), chunks))
    dt = time.perf_counter() - t0
    ranges = sample_ranges(cfg, n, desc)
    where = (f"first {n} of {total_envs} envs (global ids 0..{n - 1})" if desc is None else
             f"{sum(k for _, k in ranges)} of {total_envs} envs: the first {ranges[0][1]} of each of the "
             f"{len(ranges)} game blocks")
    return steps / dt, cores, f"{where}, {cores} threads, {dt:.2f} s"


def cpu_model():
    try:
        with open("/proc/cpuinfo") as f:
            for line in f:
                if line.startswith("model name"):
                    return line.split(":", 1)[1].strip()
    except OSError:
        pass
    return "unknown"


def cpu_oracle_single_thread(cfg, seconds, desc=None):
    """The same oracle on one host thread (about `seconds`): steps/s and sample."""
    import numpy as np

    from oracle import games as OG

    def run(n):
        steps = 0
        for off, k in sample_ranges(cfg, n, desc):
            if desc is not None:
                _, p = OG.rollout_mixed(desc[off:off + k], cfg.seed, env_offset=off)
            else:
                gid = cfg.game if cfg.game != 7 else 7 | (cfg.line << 8) | (cfg.flags << 12)
                _, p, _ = OG.rollout_start(gid, cfg.rows, cfg.cols, k, cfg.seed, env_offset=off)
            steps += int(p.astype(np.int64).sum())
        return steps

    t0 = time.perf_counter()
    run(128 if desc is None else 384)
    per_env = max((time.perf_counter() - t0) / (128 if desc is None else 384), 1e-7)
    n = int(min(cfg.num_envs, max(128, seconds / per_env)))
    t0 = time.perf_counter()
    steps = run(n)
    dt = time.perf_counter() - t0
    return steps / dt, f"{n} envs as in the multi-thread sample, 1 thread, {dt:.2f} s"


# ------------------------------------------------------------- GPU parts --
def D_shard(rank, n):
    from paper_2506_22609_b300 import dist as D

    return D.shard_offset(rank, n)


def flush_l2(buf):
    buf.add_(1)  # 256 MiB read + write: evicts the 126 MB L2


def time_steps(fn, steps, warmup, flush_buf, stream):
    import torch

    for _ in range(warmup):
        fn()
    torch.cuda.synchronize()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
    torch.cuda.nvtx.range_push("bench_timed_steps")  # the library's own calls nest inside as their C-ABI names
    for a, b in ev:
        flush_l2(flush_buf)
        a.record(stream)
        fn()
        b.record(stream)
    torch.cuda.nvtx.range_pop()
    torch.cuda.synchronize()
    return [a.elapsed_time(b) for a, b in ev]


# Outcome statistics of the last timed launch (set by bench_rollout_config and
# bench_mixed, read into the JSON line): wins of P1 and P2, draws, capped
# games (which a correct kernel never produces) and the mean game length.
LAST_OUTCOMES = {}


def note_outcomes(out, plies):
    import torch

    o = out.to(torch.int64)
    n = o.numel()
    LAST_OUTCOMES.clear()
    LAST_OUTCOMES.update({"p1_wins": int((o == 1).sum().item()), "p2_wins": int((o == 2).sum().item()),
                          "draws": int((o == 0).sum().item()), "other": int(((o < 0) | (o > 2)).sum().item()),
                          "mean_plies": round(float(plies.to(torch.float64).mean().item()), 4), "games": n})


def source_fingerprint():
    """SHA-256 over the library's sources, the header, the Python package and
    this script (the GPU machine's copy of the repository has no git history)."""
    import glob
    import hashlib

    h = hashlib.sha256()
    files = sorted(glob.glob(os.path.join(ROOT, "paper_2506_22609_b300", "csrc", "*")) +
                   glob.glob(os.path.join(ROOT, "paper_2506_22609_b300", "*.py")) +
                   [os.path.join(ROOT, "include", "ludax.h"), os.path.abspath(__file__)])
    for f in files:
        h.update(os.path.relpath(f, ROOT).encode())
        with open(f, "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def bench_rollout_config(L, W, cfg, steps, warmup, flush_buf, rank=0):
    """Fused playout of one single-game config; returns a dict of numbers."""
    import torch

    n = cfg.num_envs
    env = L.Env(cfg.game, cfg.rows, cfg.cols, n, env_offset=D_shard(rank, n), line=cfg.line, flags=cfg.flags)
    lc = L.make_cfg(*W.bench_cfg(cfg))
    out = torch.empty(n, dtype=torch.int8, device="cuda")
    plies = torch.empty(n, dtype=torch.int16, device="cuda")
    stream = torch.cuda.current_stream()
    fn = lambda: L.ludax_rollout(env.handle, cfg.seed, L.LUDAX_ROLLOUT_FROM_START, None, out, plies, lc)  # noqa: E731
    ms = time_steps(fn, steps, warmup, flush_buf, stream)
    steps_per_launch = int(plies.to(torch.int64).sum().item())
    note_outcomes(out, plies)
    return env, lc, ms, steps_per_launch


def e2e_rollout(L, cfg, steps, warmup, rank=0):
    """Public-API path with host buffers, every step: ludax_rollout_host (the
    C-ABI call with host buffers: H2D copy of the start positions in the
    packed state view -- two bits per cell plus a meta word per env --, load,
    playouts, D2H copy of outcome and plies into pinned host memory).  Six
    envs on six streams rotate, so the copies of one step overlap the
    playouts of another and the host runs up to five steps ahead (it waits
    for step i - 5 after issuing step i); the wall clock covers all steps."""
    import numpy as np
    import torch

    from paper_2506_22609_b300 import workloads as W

    n = cfg.num_envs
    cells = cfg.rows * cfg.cols
    lc = L.make_cfg(*W.bench_cfg(cfg))
    probe = L.Env(cfg.game, cfg.rows, cfg.cols, n, line=cfg.line, flags=cfg.flags)
    sp, sm = (t.cpu() for t in probe.get_state_bits())  # the game's own start rule, packed
    probe.close()
    total = sp.numel() * 8 + sm.numel() * 4
    slots, depth = [], 6
    for _ in range(depth):
        stream = torch.cuda.Stream()
        env = L.Env(cfg.game, cfg.rows, cfg.cols, n, env_offset=D_shard(rank, n), stream=stream, line=cfg.line,
                    flags=cfg.flags)
        h_planes, h_meta = sp.clone().pin_memory(), sm.clone().pin_memory()
        h_out = torch.empty(n, dtype=torch.int8).pin_memory()
        h_plies = torch.empty(n, dtype=torch.int16).pin_memory()
        slots.append((stream, env, h_planes, h_meta, h_out, h_plies))

    def launch(i):
        stream, env, h_planes, h_meta, h_out, h_plies = slots[i % depth]
        L.ludax_rollout_host(env.handle, h_planes, h_meta, cfg.seed, h_out, h_plies, lc)

    def run(k):
        for i in range(k):
            launch(i)
            if i >= depth - 1:
                slots[(i - depth + 1) % depth][0].synchronize()  # the results of step i - depth + 1 are on the host
        torch.cuda.synchronize()

    run(warmup)
    torch.cuda.synchronize()
    times = []
    for _ in range(5):  # the host and its PCIe link are shared: the median of five blocks of `steps`
        t0 = time.perf_counter()
        run(steps)
        times.append((time.perf_counter() - t0) / steps)
    dt = statistics.median(times)
    steps_per_launch = int(slots[(steps - 1) % depth][5].numpy().astype(np.int64).sum())
    # the host link alone: the same four copies per step (two up, two down), each direction timed
    # by CUDA events on its own, median of 10 after 3 warm-ups
    stream, _, h_planes, h_meta, h_out, h_plies = slots[0]
    d_planes, d_meta = torch.empty_like(h_planes, device="cuda"), torch.empty_like(h_meta, device="cuda")
    d_out, d_plies = torch.empty_like(h_out, device="cuda"), torch.empty_like(h_plies, device="cuda")

    def copy_time(fn):
        ts = []
        for i in range(13):
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            with torch.cuda.stream(stream):
                a.record()
                fn()
                b.record()
            b.synchronize()
            if i >= 3:
                ts.append(a.elapsed_time(b))
        return statistics.median(ts)

    link = {"h2d_ms": copy_time(lambda: (d_planes.copy_(h_planes, non_blocking=True),
                                         d_meta.copy_(h_meta, non_blocking=True))),
            "d2h_ms": copy_time(lambda: (h_out.copy_(d_out, non_blocking=True),
                                         h_plies.copy_(d_plies, non_blocking=True)))}
    for sl in slots:
        sl[1].close()
    return steps_per_launch / dt, total, n * 1 + n * 2, dt, cells, link, steps_per_launch


def bench_mixed(L, W, steps, warmup, flush_buf, rank=0):
    """The graph-captured mixed plan over the 2^20-env six-game batch; returns
    the per-launch times, the plies of one launch and those plies per game id."""
    import torch

    d = torch.from_numpy(W.mixed_descriptors(W.MIXED_ENVS, "block")).cuda()
    plan = L.ludax_mixed_plan_create(d, D_shard(rank, W.MIXED_ENVS), L.make_cfg(*W.mixed_bench_cfg()))
    out = torch.empty(W.MIXED_ENVS, dtype=torch.int8, device="cuda")
    plies = torch.empty(W.MIXED_ENVS, dtype=torch.int16, device="cuda")
    fn = lambda: L.ludax_mixed_plan_launch(plan, W.MIXED_SEED, out, plies)  # noqa: E731
    ms = time_steps(fn, steps, warmup, flush_buf, torch.cuda.current_stream())
    total = int(plies.to(torch.int64).sum().item())
    per_game = torch.bincount((d & 0xFF).long(), weights=plies.double()).cpu().tolist()
    note_outcomes(out, plies)
    L.ludax_mixed_plan_destroy(plan)
    return ms, total, {g: int(v) for g, v in enumerate(per_game) if v}


def e2e_mixed(L, W, steps, warmup, rank=0, depth=4):
    """Public-API path with host buffers, every step: one
    ludax_mixed_plan_launch_host call -- the 2^20 descriptors copied from
    pinned host memory, the game-grouped queue rebuilt on the device, the
    playouts, outcome and plies copied back to pinned host memory.  `depth`
    plans on their own streams rotate, so one step's copies overlap another's
    playouts; the host waits for step i - depth + 1 after issuing step i."""
    import numpy as np
    import torch

    n = W.MIXED_ENVS
    d = W.mixed_descriptors(n, "block")
    dd = torch.from_numpy(d).cuda()
    slots = []
    for _ in range(depth):
        stream = torch.cuda.Stream()
        plan = L.ludax_mixed_plan_create(dd, D_shard(rank, n), L.make_cfg(*W.mixed_bench_cfg()), stream=stream)
        slots.append((stream, plan, torch.from_numpy(d.copy()).pin_memory(),
                      torch.empty(n, dtype=torch.int8).pin_memory(), torch.empty(n, dtype=torch.int16).pin_memory()))

    def run(k):
        for i in range(k):
            _, plan, h_desc, h_out, h_plies = slots[i % depth]
            L.ludax_mixed_plan_launch_host(plan, W.MIXED_SEED, h_desc, h_out, h_plies)
            if i >= depth - 1:
                L.ludax_mixed_plan_sync(slots[(i - depth + 1) % depth][1])
        for sl in slots:
            L.ludax_mixed_plan_sync(sl[1])

    run(warmup)
    times = []
    for _ in range(3):  # the host and its link are shared: the median of three blocks of `steps`
        t0 = time.perf_counter()
        run(steps)
        times.append((time.perf_counter() - t0) / steps)
    dt = statistics.median(times)
    spl = int(slots[(steps - 1) % depth][4].numpy().astype(np.int64).sum())
    # the host link alone: the same three copies, each direction timed by CUDA events
    stream, _, h_desc, h_out, h_plies = slots[0]
    d_desc = torch.empty_like(h_desc, device="cuda")
    d_out, d_plies = torch.empty_like(h_out, device="cuda"), torch.empty_like(h_plies, device="cuda")

    def copy_time(fn):
        ts = []
        for i in range(13):
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            with torch.cuda.stream(stream):
                a.record()
                fn()
                b.record()
            b.synchronize()
            if i >= 3:
                ts.append(a.elapsed_time(b))
        return statistics.median(ts)

    link = {"h2d_ms": copy_time(lambda: d_desc.copy_(h_desc, non_blocking=True)),
            "d2h_ms": copy_time(lambda: (h_out.copy_(d_out, non_blocking=True),
                                         h_plies.copy_(d_plies, non_blocking=True)))}
    for sl in slots:
        L.ludax_mixed_plan_destroy(sl[1])
    return spl / dt, 4 * n, 3 * n, dt, link, spl, [round(t * 1e3, 4) for t in times]


SWEEP_GAMES = ("ttt", "c4", "othello", "hex11", "gomoku", "pente", "yavalath", "line_c5", "wolf_sheep", "draughts",
               "hasami_shogi")


def bench_batch_sweep(L, W, flush_buf, sizes=tuple(1 << k for k in range(10, 23, 2)), steps=8, warmup=2):
    """Throughput against batch size (Fig. 2's log-scale batch axis): fused
    playouts from the start position of every single-game workload at 2^10 ..
    2^22 envs, each timed as the median of `steps` launches after `warmup`,
    with the workload's launch shape and the L2 flushed between launches."""
    import dataclasses

    out = {}
    for name in SWEEP_GAMES:
        base = workload_cfg(name)
        row = {}
        for n in sizes:
            cfg = dataclasses.replace(base, num_envs=n, name=base.name)
            env, lc, ms, spl = bench_rollout_config(L, W, cfg, steps, warmup, flush_buf)
            env.close()
            m = statistics.median(ms)
            row[str(n)] = {"env_steps_per_s": round(spl / (m / 1e3), 1), "median_launch_ms": round(m, 5)}
        out[name] = row
    return out


def bench_compiled_library(L, steps, warmup, flush_buf, n=1 << 20, seed=3):
    """A mixed batch of every game description in the package's library,
    compiled to descriptors (env e plays library game e mod G), through the
    graph-captured mixed plan with the autotuned launch shape."""
    import numpy as np
    import torch

    from paper_2506_22609_b300 import dsl

    descs = [dsl.descriptor(t) for t in dsl.library().values()]
    d = torch.from_numpy(np.array(descs, np.int32)[np.arange(n) % len(descs)]).cuda()
    cfg, _, _ = L.ludax_autotune(d, seed, reps=3)
    plan = L.ludax_mixed_plan_create(d, 0, cfg)
    out = torch.empty(n, dtype=torch.int8, device="cuda")
    plies = torch.empty(n, dtype=torch.int16, device="cuda")
    fn = lambda: L.ludax_mixed_plan_launch(plan, seed, out, plies)  # noqa: E731
    ms = time_steps(fn, steps, warmup, flush_buf, torch.cuda.current_stream())
    total = int(plies.to(torch.int64).sum().item())
    L.ludax_mixed_plan_destroy(plan)
    m = statistics.median(ms)
    return {"env_steps_per_s": round(total / (m / 1e3), 1), "median_launch_ms": round(m, 4),
            "env_steps_per_launch": total, "games": len(descs), "num_envs": n,
            "launch": {k: getattr(cfg, k) for k in ("block_threads", "blocks_per_sm", "envs_per_thread",
                                                     "hex_nbr_table", "compact_every")}}


def bench_gavel(matches=100, iters=100, weak_iters=50):
    """App. F's GAVEL-like evaluation of every game in the package's library
    (matches between UCT agents: equal agents, then the stronger agent in
    each seat against a weaker one), all games in one launch; beside it, as
    this measurement's CPU baseline, the oracle's time for one Connect Four
    match between the same agents (one host thread, a bounded sample of 4
    matches)."""
    from oracle import games as OG
    from paper_2506_22609_b300 import dsl, gavel

    lib = dsl.library()
    gavel.evaluate_many({"warm": lib["tic_tac_toe"]}, 4, 8, 4, 0)
    r = gavel.evaluate_many(lib, matches, iters, weak_iters, 0)
    secs = r.pop("_seconds")
    searches = sum(v["searches"] for v in r.values())
    scores = {k: round(v["gavel_score"], 3) for k, v in sorted(r.items())}
    t0 = time.perf_counter()
    OG.mcts_play(1, 6, 7, 4, 0, iters, iters)
    cpu_c4 = (time.perf_counter() - t0) / 4
    return {"seconds": round(secs, 4), "games": len(r), "matches": len(r) * (matches + matches), "iters": iters,
            "weak_iters": weak_iters, "searches": searches, "searches_per_s": round(searches / secs, 1),
            "iterations_per_s_lower_bound": round(searches * weak_iters / secs, 1), "gavel_scores": scores,
            "median_gavel_score": round(float(statistics.median(scores.values())), 3),
            "interesting": sorted(k for k, v in r.items() if v["interesting"]),
            "cpu_baseline": {"kind": "oracle", "unit": "s per Connect Four match",
                             "value": round(cpu_c4, 4), "cores": 1,
                             "sample": "4 Connect Four matches between 100-iteration agents, one host thread"}}


# algorithmic bytes of one env step in step-per-launch mode: read two planes
# and the meta word (20 B), write them back (20 B), rewards (8 B), terminated (1 B)
STEP_BYTES_PER_ENV = 49


def bench_step_workload(L, steps, warmup, flush_buf, rank=0, n=1 << 24):
    """Timed step = one ludax_random_step over n Connect Four envs, each step
    taken on a batch reset and advanced 4 plies outside the timed events."""
    import torch

    env = L.Env("c4", 6, 7, n, env_offset=D_shard(rank, n))
    rew = torch.empty(n, 2, device="cuda")
    term = torch.empty(n, dtype=torch.uint8, device="cuda")

    def prepare():
        L.ludax_reset(env.handle)
        for _ in range(4):
            L.ludax_random_step(env.handle, 1, rew, term)

    stream = torch.cuda.current_stream()
    for _ in range(warmup):
        prepare()
        L.ludax_random_step(env.handle, 1, rew, term)
    torch.cuda.synchronize()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
    for a, b in ev:
        prepare()
        flush_l2(flush_buf)
        a.record(stream)
        L.ludax_random_step(env.handle, 1, rew, term)
        b.record(stream)
    torch.cuda.synchronize()
    env.close()
    return [a.elapsed_time(b) for a, b in ev], n, n


def bench_step_mode(L, steps, flush_buf, game="c4", n=1 << 24):
    """Step-per-launch mode (ludax_random_step) at a batch far above L2:
    HBM-bound; returns achieved GB/s of algorithmic state traffic."""
    import torch

    rows, cols = {"c4": (6, 7), "othello": (8, 8)}[game]
    env = L.Env(game, rows, cols, n)
    rew = torch.empty(n, 2, device="cuda")
    term = torch.empty(n, dtype=torch.uint8, device="cuda")
    # advance a few plies so that the timed steps are mid-game
    for _ in range(4):
        L.ludax_random_step(env.handle, 2, rew, term)
    ms = time_steps(lambda: L.ludax_random_step(env.handle, 2, rew, term), steps, 2, flush_buf,
                    torch.cuda.current_stream())
    # per env-step: read 2 planes + meta (20 B), write 2 planes + meta (20 B), rewards 8 B, terminated 1 B
    bytes_per = 20 + 20 + 8 + 1
    t = statistics.median(ms) / 1e3
    env.close()
    return {"workload": f"{game}_{n}env_random_step", "ms": statistics.median(ms),
            "gbs": n * bytes_per / t / 1e9, "bytes_per_env_step": bytes_per, "env_steps_per_s": n / t}


def bench_dense(L, peaks, flush_buf, M=65536, N=512, K=512):
    """The value net's hidden layer (M x N x K BF16 -> FP32 -> bias, ReLU, BF16)
    on the tcgen05 kernel, and the full net forward on both tensor paths."""
    import torch

    g = torch.Generator(device="cuda").manual_seed(0)
    a = (torch.randn(M, K, device="cuda", generator=g) * 0.5).to(torch.bfloat16).view(torch.int16)
    b = (torch.randn(N, K, device="cuda", generator=g) * 0.05).to(torch.bfloat16).view(torch.int16)
    bias = torch.zeros(N, device="cuda")
    out = torch.empty(M, N, dtype=torch.int16, device="cuda")
    ms = time_steps(lambda: L.ludax_dense_bf16_relu(a, b, bias, out), 20, 3, flush_buf, torch.cuda.current_stream())
    t = statistics.median(ms) / 1e3
    tflops = 2.0 * M * N * K / t / 1e12
    res = {"shape": [M, N, K], "median_ms": round(t * 1e3, 4), "tflops": round(tflops, 1),
           "frac_of_bf16_peak": round(tflops / float(peaks.get("bf16_tflops", 1800.0)), 4),
           "device_error": L.ludax_device_error()}
    net = L.Net(64, M)
    x = torch.zeros(M, net.in_pad, dtype=torch.int16, device="cuda")
    flops = 2.0 * M * (net.in_pad * 512 + 512 * 512 + 512)
    for path, name in ((1, "tcgen05_one_launch"), (2, "tcgen05_two_launches"), (0, "mma_sync")):
        net.set_tensor_path(path)
        msf = time_steps(lambda: net.forward(x), 10, 2, flush_buf, torch.cuda.current_stream())
        tf = statistics.median(msf) / 1e3
        res["net_forward_" + name] = {"median_ms": round(tf * 1e3, 4), "tflops": round(flops / tf / 1e12, 1)}
    net.close()
    return res


def bench_train_step(L, peaks, flush_buf, steps=20, warmup=3, B=65536):
    """One Adam step of the value net (forward with labels, backward, Adam)
    on a 65,536-row batch of Othello (129 inputs) and Hex 11 (243 inputs)
    rows, on the tcgen05 path and on the mma.sync path; the rows hold a
    stone in 30% of the cells.  FLOPs per step as the tcgen05 kernels run
    them: layer 1 over the input columns up to the next multiple of 64 (k1:
    Othello 192, Hex 11 256), layer 2, the head, dZ1, dW2 and dW1 (over all
    in_pad columns): 2 B (512 (k1 + in_pad) + 3 * 512 * 512 + 512)."""
    import torch

    from paper_2506_22609_b300 import workloads as W

    out = {}
    g = torch.Generator(device="cuda").manual_seed(3)
    for game, cells in (("othello", 64), ("hex11", 121)):
        net = L.Net(cells, B)
        net.set_params(torch.from_numpy(W.init_params(cells, 1)).cuda())
        x = (torch.rand(B, net.in_pad, device="cuda", generator=g) < 0.3).to(torch.bfloat16)
        x[:, 2 * cells + 1:] = 0
        xb, yb = x.view(torch.int16), torch.rand(B, device="cuda", generator=g)
        k1 = min(net.in_pad, (2 * cells + 1 + 63) // 64 * 64)
        flops = 2.0 * B * (512 * (k1 + net.in_pad) + 3 * 512 * 512 + 512)
        # HBM bytes of the tcgen05 step's dataflow (BF16 activations): X read by layer 1 (k1
        # columns) and dW1 (in_pad); H1 written by the forward (which reads it back for layer 2
        # from L2, within the launch) and read by dW2, and its non-zero bits (64 B per row)
        # written by the forward and read by dZ1 as its mask; H2 written and read by the head's
        # backward; dZ2 written and read by dZ1 and dW2; dZ1 written (its column sums are taken
        # in the same epilogue) and read by dW1; the finish kernel reads and writes parameters and
        # both Adam moments and writes the BF16 weight copies (~7 FP32 words per parameter).  The
        # mma.sync path reads H1 itself for the mask (another 1 KB per row).
        nbytes = 2.0 * B * (k1 + net.in_pad + 512 * (2 + 2 + 3 + 2)) + 2.0 * 64 * B + 4.0 * 7 * net.num_params
        res = {"batch": B, "in_pad": net.in_pad, "layer1_columns": k1, "gflop_per_step": round(flops / 1e9, 2),
               "alg_mbytes_per_step": round(nbytes / 1e6, 1),
               "arithmetic_intensity_flop_per_byte": round(flops / nbytes, 1)}
        for path, name in ((1, "tcgen05"), (0, "mma_sync")):
            net.set_tensor_path(path)
            ms = time_steps(lambda: net.train_step(xb, yb, 1e-3), steps, warmup, flush_buf,
                            torch.cuda.current_stream())
            t = statistics.median(ms) / 1e3
            tf = flops / t / 1e12
            gbs = nbytes / t / 1e9
            res[name] = {"median_ms": round(t * 1e3, 4), "steps_per_s": round(1 / t, 1), "tflops": round(tf, 1),
                         "frac_of_bf16_peak": round(tf / float(peaks.get("bf16_tflops", 1800.0)), 4),
                         "hbm_gbs": round(gbs, 1), "frac_of_hbm": round(gbs / float(peaks.get("hbm_gbs", 6400.0)), 4)}
        res["device_error"] = L.ludax_device_error()
        net.close()
        out[game] = res
    return out


def bench_valuenet(seeds=(5, 6, 7)):
    """The learned part: 2M training positions per game, 65,536 validation
    positions (which choose the epoch, K and M) and 100k held-out positions
    (evaluated once); value estimates/s of the truncated estimator (8 random
    plies, then the net) and of full playouts at MAE <= 0.05 against a
    256-playout reference, over several seeds (mean and sd of each seed's
    held-out numbers)."""
    from paper_2506_22609_b300 import valuenet as V

    def spread(xs):
        return {"mean": round(statistics.mean(xs), 5), "sd": round(statistics.stdev(xs), 5) if len(xs) > 1 else 0.0,
                "values": [round(x, 5) for x in xs]}

    out = {}
    for game in ("othello", "hex11"):
        runs = [V.run(game, seed=sd) for sd in seeds]
        ev = [r["eval"] for r in runs]
        out[game] = {
            "seeds": list(seeds),
            "selected_K": [r["validation"]["K"] for r in runs], "selected_M": [r["validation"]["M"] for r in runs],
            "epoch_kept": [r["epoch_kept"] for r in runs],
            "truncated_mae": spread([e["truncated_selected"]["mae"] for e in ev]),
            "truncated_estimates_per_s": spread([e["truncated_selected"]["estimates_per_s"] for e in ev]),
            "full_mae": spread([e["full_selected"]["mae"] for e in ev]),
            "full_estimates_per_s": spread([e["full_selected"]["estimates_per_s"] for e in ev]),
            "gain_estimates_per_s": spread([e["gain_estimates_per_s"] for e in ev]),
            "equal_mae": ev[0]["equal_mae"], "equal_time": ev[0]["equal_time"],
            "net_only_mae": spread([e["net_only_mae"] for e in ev]),
            "reference_noise_mae": round(ev[0]["reference_noise_mae"], 5), "target_mae": ev[0]["target_mae"],
            "validation_truncated": runs[0]["validation"]["truncated"],
            "all_truncated": ev[0]["truncated"], "all_full": ev[0]["full_playouts"],
            "train_seconds": [round(r["train_seconds"], 3) for r in runs],
            "train_steps": [r["train_steps"] for r in runs], "data_seconds": round(runs[0]["data_seconds"], 3),
            "n_train": runs[0]["n_train"], "n_val": runs[0]["n_val"], "n_eval": runs[0]["n_eval"],
            "inference_rows": ev[0]["inference_rows"]}
    return out


def bench_threads_per_env(L, sizes=(7, 9, 11), batches=(1024, 4096, 16384, 65536, 174763), seed=4, reps=3):
    """The single-game autotuner over Hex boards and batch sizes, reduced to
    the fastest launch shape for each threads-per-env value (1, 2, 4): ms
    per launch from the start position and env steps per second."""
    out = {}
    for size in sizes:
        for n in batches:
            env = L.Env("hex", size, size, n)
            best, best_ms, table = L.ludax_autotune_env(env.handle, seed, reps=reps)
            per = {}
            for c, ms in table:
                t = max(1, c.threads_per_env)
                if t not in per or ms < per[t][1]:
                    per[t] = (c.as_dict(), ms)
            _, plies = env.rollout(seed, cfg=best)
            spl = int(plies.to(dtype=__import__("torch").int64).sum().item())
            out[f"hex{size}_{n}env"] = {str(t): {"ms": round(v[1], 4), "env_steps_per_s": round(spl / (v[1] / 1e3), 1),
                                                 "launch": v[0]} for t, v in sorted(per.items())}
            env.close()
    return out


def bench_lanes_per_warp(L, batches=(1024, 4096, 16384, 65536), seed=4, reps=3):
    """The single-game autotuner over games and small batch sizes, reduced to
    the fastest one-lane-per-env shape for each lanes-per-warp value (32 =
    full warps, 16, 8): ms per launch from the start position and env steps
    per second."""
    import torch

    games = (("ttt", 3, 3), ("c4", 6, 7), ("othello", 8, 8), ("hex", 7, 7), ("hex", 11, 11))
    out = {}
    for game, rows, cols in games:
        for n in batches:
            env = L.Env(game, rows, cols, n)
            best, best_ms, table = L.ludax_autotune_env(env.handle, seed, reps=reps)
            per = {}
            for c, ms in table:
                if c.threads_per_env > 1:
                    continue
                lanes = c.lanes_per_warp or 32
                if lanes not in per or ms < per[lanes][1]:
                    per[lanes] = (c.as_dict(), ms)
            _, plies = env.rollout(seed, cfg=best)
            spl = int(plies.to(dtype=torch.int64).sum().item())
            out[f"{game}{rows}x{cols}_{n}env"] = {
                str(k): {"ms": round(v[1], 4), "env_steps_per_s": round(spl / (v[1] / 1e3), 1), "launch": v[0]}
                for k, v in sorted(per.items(), reverse=True)}
            env.close()
    return out


def bench_int_peak(L, iters=1 << 16):
    """What a stream of one integer op reaches (LOP3, IADD, SHF, IMAD,
    IMAD.HI, and LOP3 + IMAD on alternate chains; 8 independent chains per
    thread, every SM fully occupied), against the issue peak (4 warp
    instructions per clock per SM) and the ALU pipe's half of it: the
    denominators of the playouts' roofline."""
    import torch

    dev = torch.cuda.current_device()
    props = torch.cuda.get_device_properties(dev)
    out = {}
    with ClockSampler(dev) as clk:
        for kind in ("lop3", "iadd", "shf", "imad", "imad_hi", "lop3_imad"):
            ms = []
            for i in range(5):
                a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                a.record()
                ops = L.ludax_int_peak(kind, iters)
                b.record()
                torch.cuda.synchronize()
                if i:
                    ms.append(a.elapsed_time(b))
            t = statistics.median(ms) / 1e3
            out[kind] = {"tops": round(ops / t / 1e12, 3), "ms": round(t * 1e3, 3), "ops": ops}
    rec = clk.record()
    mhz = rec["sm_mhz"] or rec["sm_max_mhz"] or 2032
    issue = props.multi_processor_count * 128 * mhz * 1e6 / 1e12
    out["clocks"] = rec
    out["issue_peak_tops"] = round(issue, 3)
    out["alu_pipe_peak_tops"] = round(issue / 2, 3)
    for kind in ("lop3", "iadd", "shf", "imad", "imad_hi", "lop3_imad"):
        out[kind]["frac_of_issue_peak"] = round(out[kind]["tops"] / issue, 3)
    return out


def bench_value_estimator(n=100_000):
    """The truncated estimator alone (8 random plies, then the net; Othello
    K = 8, Hex 11 K = 1, the continuation counts that reach MAE 0.05 with the
    trained net) on n sampled positions with an untrained net of the same
    shape: its speed does not depend on the weights.  A small case for
    profilers; value_net measures the same path after training."""
    import torch

    from paper_2506_22609_b300 import ludax as L
    from paper_2506_22609_b300 import valuenet as V
    from paper_2506_22609_b300 import workloads as W

    out = {}
    for game, K in (("othello", 8), ("hex11", 1)):
        g, rows, cols = V.GAMES[game]
        env, _ = V.sample_positions(g, rows, cols, n, 5, 0)
        net = L.Net(rows * cols, 65536)
        net.set_params(torch.from_numpy(W.init_params(rows * cols, 5)).cuda())
        inet, owned = V.inference_net(net, n * K)
        val = torch.empty(n, dtype=torch.float32, device="cuda")
        _, dt = V.cuda_time_median(lambda: L.ludax_truncated_value(env.handle, inet.handle, 77, K, 8, val))
        out[game] = {"K": K, "plies": 8, "positions": n, "rows": n * K, "seconds": dt, "estimates_per_s": n / dt}
        if owned:
            inet.close()
        net.close()
        env.close()
    return out


# ------------------------------------------------------------------ main --
def main():
    args = parse()
    from paper_2506_22609_b300 import dist as D

    rank, world, local = D.world_info()

    if args.impl == "reference":
        if rank != 0:
            return 0
        return reference_arm(args)

    import torch

    from paper_2506_22609_b300 import build as B

    B.build()
    from paper_2506_22609_b300 import ludax as L
    from paper_2506_22609_b300 import workloads as W

    torch.cuda.set_device(local)
    if world > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    peaks, peak_kind = measured_peaks()
    flush_buf = torch.zeros(64 << 20, dtype=torch.float32, device="cuda")  # 256 MiB
    if args.only:
        if args.only == "dense_layer":
            res = bench_dense(L, peaks, flush_buf)
        elif args.only == "gavel_library":
            res = bench_gavel()
        elif args.only == "value_net":
            res = bench_valuenet()
        elif args.only == "value_estimator":
            res = bench_value_estimator()
        elif args.only == "int_peak":
            res = bench_int_peak(L)
        elif args.only == "train_step":
            res = bench_train_step(L, peaks, flush_buf, max(args.steps, 5), args.warmup)
        elif args.only == "threads_per_env":
            res = bench_threads_per_env(L)
        elif args.only == "lanes_per_warp":
            res = bench_lanes_per_warp(L)
        else:
            res = bench_batch_sweep(L, W, flush_buf)
        if rank == 0:
            print(json.dumps({args.only: res}), flush=True)
        return 0

    cfg = workload_cfg(args.workload) if args.workload not in ("mixed", "step_c4") else None
    with ClockSampler(local) as clk:
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize()
        if args.workload == "step_c4":
            ms, steps_per_launch, n_envs = bench_step_workload(L, args.steps, args.warmup, flush_buf, rank)
            wl_name, seed, launch = "connect4_6x7_16777216env_random_step_seed1", 1, {"block_threads": 256}
        elif cfg is not None:
            env, lc, ms, steps_per_launch = bench_rollout_config(L, W, cfg, args.steps, args.warmup, flush_buf, rank)
            wl_name, n_envs, seed = cfg.name, cfg.num_envs, cfg.seed
            launch = lc.as_dict()
        else:
            ms, steps_per_launch, plies_per_game = bench_mixed(L, W, args.steps, args.warmup, flush_buf, rank)
            wl_name, n_envs, seed = "mixed6_1048576env_seed3_graph", W.MIXED_ENVS, W.MIXED_SEED
            launch = dict(zip(("block_threads", "blocks_per_sm", "envs_per_thread", "hex_nbr_table",
                               "compact_every"), W.mixed_bench_cfg()))
        torch.cuda.synchronize()
        if world > 1:
            dist.barrier()
    clocks = clk.record()

    total_ms, all_steps = D.aggregate(sum(ms), steps_per_launch, device="cuda")
    value = all_steps * args.steps / (total_ms / 1e3)

    # roofline of the fused playout kernel: integer issue
    sms = torch.cuda.get_device_properties(local).multi_processor_count
    max_mhz = float(peaks.get("sm_max_mhz", 2032.0))
    peak_ops = sms * 128 * max_mhz * 1e6  # 32-bit lanes x clock
    ops_prior = None
    if cfg is not None and game_key(cfg) in ALG_OPS_PER_STEP:
        ops_per_launch = ALG_OPS_PER_STEP[game_key(cfg)] * steps_per_launch
        if game_key(cfg) in PRIOR_OPS_PER_STEP:
            ops_prior = PRIOR_OPS_PER_STEP[game_key(cfg)] * steps_per_launch
    elif args.workload == "mixed":
        # the sum over the mix's games of (ops per step x that game's plies in the launch)
        ops_per_launch = sum(ALG_OPS_PER_STEP[GAME_KEYS[g]] * v for g, v in plies_per_game.items())
        ops_prior = sum(PRIOR_OPS_PER_STEP[GAME_KEYS[g]] * v for g, v in plies_per_game.items())
    else:
        ops_per_launch = None
    med = statistics.median(ms)
    roofline = None
    if args.workload == "step_c4":
        bytes_per = STEP_BYTES_PER_ENV
        achieved = n_envs * bytes_per / (med / 1e3) / 1e9
        peak = float(peaks.get("hbm_gbs", 6400.0))
        roofline = {"bound": "hbm", "achieved": round(achieved, 1), "peak": peak, "unit": "GB/s",
                    "frac": round(achieved / peak, 4), "traffic": NCU_TRAFFIC_BYTES.get(wl_name),
                    "peak_source": f"hbm_gbs ({peak_kind})", "alg_bytes_per_env_step": bytes_per,
                    "median_launch_ms": round(med, 5)}
    if ops_per_launch:
        # frac uses the prior estimates of the op counts where they exist; the
        # counts of the bitboard algorithm and ncu's executed count sit beside it
        alu_pipe = peak_ops / 2  # logic/shift/add run on the ALU pipe: 64 lanes per clock per SM
        achieved_b = ops_per_launch / (med / 1e3) / 1e12
        achieved = (ops_prior or ops_per_launch) / (med / 1e3) / 1e12
        if cfg is not None:
            per_step = {"builder": ALG_OPS_PER_STEP[game_key(cfg)],
                        "prior_estimate": PRIOR_OPS_PER_STEP.get(game_key(cfg))}
        else:
            per_step = {"builder": {GAME_KEYS[g]: ALG_OPS_PER_STEP[GAME_KEYS[g]] for g in plies_per_game},
                        "prior_estimate": {GAME_KEYS[g]: PRIOR_OPS_PER_STEP[GAME_KEYS[g]] for g in plies_per_game},
                        "plies_per_game": {GAME_KEYS[g]: v for g, v in plies_per_game.items()}}
        roofline = {"bound": "alu", "achieved": round(achieved, 3), "peak": round(peak_ops / 1e12, 3),
                    "unit": "Tops/s (32-bit integer)", "frac": round(achieved / (peak_ops / 1e12), 4),
                    "counts": "prior_estimate" if ops_prior else "builder",
                    "alu_pipe_peak": round(alu_pipe / 1e12, 3), "alu_pipe_frac": round(achieved / (alu_pipe / 1e12), 4),
                    "frac_builder_counts": round(achieved_b / (peak_ops / 1e12), 4),
                    "ncu_thread_instructions_per_step": NCU_THREAD_INST_PER_STEP.get(wl_name),
                    "traffic": NCU_TRAFFIC_BYTES.get(wl_name),
                    "peak_source": f"{sms} SMs x 128 int32 lanes x {max_mhz:.0f} MHz (sm_max_mhz, {peak_kind})",
                    "alg_ops_per_step": per_step, "median_launch_ms": round(med, 5)}

    line = {"metric": METRIC, "value": round(value, 1), "unit": "env steps/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(total_ms / args.steps, 5),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u64",
            "data": "synthetic (start positions; counter-based uniform-random policy)",
            "config": {"workload": wl_name, "num_envs_per_gpu": n_envs, "seed": seed, "launch": launch,
                       "l2": "flushed between steps (256 MiB write outside the timed events)",
                       "timing": "CUDA events around each launch on the launching stream, summed over steps",
                       "env_steps_per_launch": steps_per_launch, "episodes_per_launch": n_envs},
            "roofline": roofline, "clocks": clocks,
            "gpu_launches": args.steps,
            "outcomes": dict(LAST_OUTCOMES),
            "run": {"source_sha256": source_fingerprint(), "gpu": torch.cuda.get_device_name(),
                    "cuda_runtime": torch.version.cuda, "torch": torch.__version__}}

    if rank == 0 and cfg is not None and args.workload != "step_c4":
        e2e_val, h2d, d2h, dt, _, link, spl = e2e_rollout(L, cfg, max(3, min(args.steps, 100)), 3, rank)
        # with the copies of one step overlapping another's playouts, a step costs at least the
        # slowest of: its uploads, its downloads, its playout launch
        t_bound = max(link["h2d_ms"], link["d2h_ms"], med) / 1e3
        line["e2e"] = {"value": round(e2e_val * world, 1), "unit": "env steps/s", "h2d_bytes_per_step": h2d,
                       "d2h_bytes_per_step": d2h, "ms_per_step": round(dt * 1e3, 4),
                       "link": {"h2d_ms": round(link["h2d_ms"], 4), "d2h_ms": round(link["d2h_ms"], 4),
                                "h2d_gbs": round(h2d / link["h2d_ms"] / 1e6, 2),
                                "d2h_gbs": round(d2h / link["d2h_ms"] / 1e6, 2),
                                "bound_env_steps_per_s": round(spl / t_bound, 1),
                                "frac": round(e2e_val / (spl / t_bound), 4)},
                       "path": "ludax_rollout_host per step: pinned host start positions in the packed state view "
                               "(2 bits per cell + a meta word per env) -> device -> playouts -> pinned host "
                               "outcome/plies; six envs on six streams rotate so one step's copies overlap "
                               "another's playouts; wall clock over blocks of steps, median of 5 blocks"}
    if rank == 0 and args.workload == "mixed":
        e2e_val, h2d, d2h, dt, link, spl, blocks = e2e_mixed(L, W, max(3, min(args.steps, 50)), 3, rank)
        t_bound = max(link["h2d_ms"], link["d2h_ms"], med) / 1e3
        line["e2e"] = {"value": round(e2e_val * world, 1), "unit": "env steps/s", "h2d_bytes_per_step": h2d,
                       "d2h_bytes_per_step": d2h, "ms_per_step": round(dt * 1e3, 4), "ms_per_step_blocks": blocks,
                       "link": {"h2d_ms": round(link["h2d_ms"], 4), "d2h_ms": round(link["d2h_ms"], 4),
                                "h2d_gbs": round(h2d / link["h2d_ms"] / 1e6, 2),
                                "d2h_gbs": round(d2h / link["d2h_ms"] / 1e6, 2),
                                "bound_env_steps_per_s": round(spl / t_bound, 1),
                                "frac": round(e2e_val / (spl / t_bound), 4)},
                       "path": "ludax_mixed_plan_launch_host per step: pinned host descriptors (int32 per env) -> "
                               "device -> work queue rebuilt on the device -> playouts -> pinned host outcome/plies; "
                               "four plans on four streams rotate so one step's copies overlap another's playouts; "
                               "wall clock over blocks of steps, median of 3 blocks"}
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        desc = None
        if args.workload == "step_c4":
            ccfg = W.C4_64K
        elif cfg is not None:
            ccfg = cfg
        else:
            ccfg, desc = W_mixed_cfg(W), W.mixed_descriptors(W.MIXED_ENVS, "block")
        v, cores, sample = cpu_oracle_rate(ccfg, args.cpu_seconds, desc=desc)
        v1, sample1 = cpu_oracle_single_thread(ccfg, min(2.0, args.cpu_seconds / 4), desc=desc)
        if args.workload == "step_c4":
            sample = "Connect Four playouts: " + sample
        line["cpu_baseline"] = {"value": round(v, 1), "unit": "env steps/s", "cores": cores, "kind": "oracle",
                                "sample": sample, "cpu_model": cpu_model(),
                                "single_thread": {"value": round(v1, 1), "sample": sample1}}
    if rank == 0 and world == 1 and not args.no_extras:
        extras = {}
        for name in ("ttt", "c4", "othello", "hex11", "gomoku", "pente", "yavalath", "line_c5", "wolf_sheep",
                     "draughts", "hasami_shogi"):
            if name == args.workload:
                continue
            c = workload_cfg(name)
            e, lc, ms2, spl = bench_rollout_config(L, W, c, 20, 3, flush_buf)
            m2 = statistics.median(ms2)
            rate = spl / (m2 / 1e3)
            extras[c.name] = {"env_steps_per_s": round(rate, 1), "median_launch_ms": round(m2, 5),
                              "env_steps_per_launch": spl, "launch": lc.as_dict(),
                              "alu_frac": (round(ALG_OPS_PER_STEP[game_key(c)] * rate / peak_ops, 4)
                                           if game_key(c) in ALG_OPS_PER_STEP else None)}
            e.close()
        if args.workload != "mixed":
            ms3, tot, _ = bench_mixed(L, W, 10, 2, flush_buf)
            m3 = statistics.median(ms3)
            extras["mixed6_1048576env_seed3_graph"] = {"env_steps_per_s": round(tot / (m3 / 1e3), 1),
                                                       "median_launch_ms": round(m3, 4), "env_steps_per_launch": tot}
        extras["compiled_library_1048576env_seed3"] = bench_compiled_library(L, 10, 2, flush_buf)
        for gname in ("c4", "othello"):
            sm = bench_step_mode(L, 10, flush_buf, gname, 1 << 24 if gname == "c4" else 1 << 22)
            sm["hbm_frac"] = round(sm["gbs"] / float(peaks.get("hbm_gbs", 6400.0)), 4)
            extras["step_mode_" + gname] = sm
        extras["dense_layer"] = bench_dense(L, peaks, flush_buf)
        extras["train_step"] = bench_train_step(L, peaks, flush_buf)
        extras["gavel_library"] = bench_gavel()
        if not args.no_valuenet:
            extras["value_net"] = bench_valuenet()
        line["extra_workloads"] = extras
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()
    return 0


def W_mixed_cfg(W):
    return W.Config("mixed6_1048576env_seed3", -1, 0, 0, W.MIXED_ENVS, W.MIXED_SEED)


def reference_arm(args):
    """The CPU oracle as the reference arm: each step is a bounded sample of
    the workload on all host cores."""
    from paper_2506_22609_b300 import workloads as W

    if args.workload == "mixed":
        cfg = W_mixed_cfg(W)
        desc = W.mixed_descriptors(W.MIXED_ENVS, "block")
    else:
        cfg, desc = workload_cfg(args.workload), None
    per_step = max(0.5, min(4.0, 120.0 / max(1, args.steps + args.warmup)))
    vals, sample = [], ""
    for i in range(args.warmup + args.steps):
        v, cores, sample = cpu_oracle_rate(cfg, per_step, desc=desc)
        if i >= args.warmup:
            vals.append(v)
    value = statistics.median(vals)
    line = {"impl": "reference", "metric": METRIC, "value": round(value, 1), "unit": "env steps/s", "n_gpus": 1,
            "steps": args.steps, "warmup": args.warmup, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "int8 cells", "data": "synthetic",
            "config": {"workload": cfg.name + ("_graph" if args.workload == "mixed" else ""),
                       "num_envs_per_gpu": cfg.num_envs, "seed": cfg.seed},
            "cpu_baseline": {"kind": "oracle", "cores": cores, "sample": sample, "value": round(value, 1),
                             "unit": "env steps/s"},
            "e2e": {"value": round(value, 1), "unit": "env steps/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


if __name__ == "__main__":
    sys.exit(main())
