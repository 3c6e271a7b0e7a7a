"""Workload definitions and seeded input generators.

This module holds no game arithmetic: it only names the benchmark
configurations (game, board, number of envs, seed) and builds the inputs that
both the CUDA path and the CPU oracle receive -- per-env game descriptors for
mixed batches and seeded action/position samples for step tests.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np

TTT, C4, OTHELLO, HEX, GOMOKU, PENTE, YAVALATH = 0, 1, 2, 3, 4, 5, 6


def desc(game: int, rows: int, cols: int) -> int:
    """Per-env descriptor: game | rows << 8 | cols << 16."""
    return game | (rows << 8) | (cols << 16)


@dataclass(frozen=True)
class Config:
    name: str
    game: int
    rows: int
    cols: int
    num_envs: int
    seed: int
    line: int = 0      # parametric line game: line length
    flags: int = 0     # parametric line game: exact / gravity / misere bits


# Uniform-random playouts from the start position (the random-policy
# benchmark of the paper's Sec. 6, at the batch sizes used here).
TTT_1K = Config("ttt3x3_1024env_seed0", TTT, 3, 3, 1024, 0)
C4_64K = Config("connect4_6x7_65536env_seed1", C4, 6, 7, 65536, 1)
OTHELLO_256K = Config("othello8x8_262144env_seed2", OTHELLO, 8, 8, 262144, 2)
HEX11_64K = Config("hex11x11_65536env_seed4", HEX, 11, 11, 65536, 4)
# the line-game family (Gomoku, Pente, Yavalath)
GOMOKU_64K = Config("gomoku15x15_65536env_seed5", GOMOKU, 15, 15, 65536, 5)
PENTE_64K = Config("pente19x19_65536env_seed6", PENTE, 19, 19, 65536, 6)
YAVALATH_64K = Config("yavalath61_65536env_seed7", YAVALATH, 9, 9, 65536, 7)

# The mixed batch: 2^20 envs over six games, seed 3.
MIXED_GAMES = [(TTT, 3, 3), (C4, 6, 7), (OTHELLO, 8, 8), (HEX, 7, 7), (HEX, 9, 9), (HEX, 11, 11)]
MIXED_ENVS = 1 << 20
MIXED_SEED = 3


def mixed_descriptors(n: int = MIXED_ENVS, layout: str = "block") -> np.ndarray:
    """Descriptors for an even split of n envs over the six mixed games.

    layout "block": env e plays game floor(6e/n) (contiguous thirds... sixths);
    layout "interleave": env e plays game e mod 6 (every warp mixes games).
    """
    e = np.arange(n, dtype=np.int64)
    g = (6 * e) // n if layout == "block" else e % 6
    table = np.array([desc(*x) for x in MIXED_GAMES], dtype=np.int32)
    return table[g]


def random_descriptors(n: int, seed: int) -> np.ndarray:
    """Descriptors drawn uniformly over every supported (game, size)."""
    all_desc = [desc(TTT, 3, 3), desc(C4, 6, 7), desc(OTHELLO, 8, 8)] + [desc(HEX, k, k) for k in range(2, 12)] + [
        desc(GOMOKU, 15, 15), desc(PENTE, 19, 19), desc(YAVALATH, 9, 9)]
    rng = np.random.default_rng(seed)
    return np.array(all_desc, dtype=np.int32)[rng.integers(0, len(all_desc), n)]


def sample_envs(n_total: int, k: int, seed: int) -> np.ndarray:
    """k distinct env indices in [0, n_total), always including both ends."""
    rng = np.random.default_rng(seed)
    idx = rng.choice(n_total, size=min(k, n_total), replace=False)
    idx[0], idx[-1] = 0, n_total - 1
    return np.unique(idx)


# Launch shapes the benchmark times (block_threads, blocks_per_sm,
# envs_per_thread, hex_nbr_table, compact_every): the fastest candidates of
# ludax_autotune_env / ludax_autotune on a B300.
# move games (action = from * cells + to), 200-ply cap
WOLF_SHEEP_64K = Config("wolf_sheep8x8_65536env_seed9", 8, 8, 8, 65536, 9)
DRAUGHTS_64K = Config("draughts8x8_65536env_seed10", 9, 8, 8, 65536, 10)
HASAMI_64K = Config("hasami_shogi9x9_65536env_seed11", 10, 9, 9, 65536, 11)

# the parametric line-game kernel: exactly five in a row, with gravity, on 9 x 12
CONNECT5_9X12_64K = Config("connect5exact_gravity_9x12_65536env_seed8", 7, 9, 12, 65536, 8, line=5, flags=3)

BENCH_CFGS = {
    TTT_1K.name: (64, 0, 1, 0, 16),
    C4_64K.name: (448, 4, 1, 0, 16),
    OTHELLO_256K.name: (448, 0, 1, 0, 0),
    HEX11_64K.name: (448, 2, 1, 1, 16),
    GOMOKU_64K.name: (448, 0, 1, 0, 16),
    PENTE_64K.name: (448, 4, 1, 0, 16),
    YAVALATH_64K.name: (448, 0, 1, 0, 16),
    CONNECT5_9X12_64K.name: (448, 0, 1, 0, 16),
    WOLF_SHEEP_64K.name: (448, 0, 1, 0, 16),
    DRAUGHTS_64K.name: (448, 0, 1, 0, 16),
    HASAMI_64K.name: (448, 2, 1, 0, 16),
}
MIXED_BENCH_CFG = (256, 0, 1, 1, 0)


def bench_cfg(cfg: Config) -> tuple:
    return BENCH_CFGS.get(cfg.name, (256, 0, 1, 0, 0))


def mixed_bench_cfg() -> tuple:
    return MIXED_BENCH_CFG


# ------------------------------------------------------------ value net --
NET_HIDDEN = 512


def net_in_pad(cells: int) -> int:
    return ((2 * cells + 1 + 127) // 128) * 128


def init_params(cells: int, seed: int) -> np.ndarray:
    """Initial flat parameter vector (float32) for the value network:
    Kaiming-uniform hidden weights (bound sqrt(6 / fan_in), fan_in counting
    the real inputs 2*cells+1), output weights uniform within 1/sqrt(512),
    zero biases.  Layout W1 [512][in_pad], b1, W2 [512][512], b2, w3, b3."""
    rng = np.random.default_rng(seed)
    H, K, kin = NET_HIDDEN, net_in_pad(cells), 2 * cells + 1
    W1 = np.zeros((H, K), np.float32)
    W1[:, :kin] = rng.uniform(-1, 1, (H, kin)) * np.sqrt(6.0 / kin)
    W2 = rng.uniform(-1, 1, (H, H)) * np.sqrt(6.0 / H)
    w3 = rng.uniform(-1, 1, H) / np.sqrt(H)
    z = np.zeros(H)
    return np.concatenate([W1.reshape(-1), z, W2.reshape(-1), z, w3, [0.0]]).astype(np.float32)


def ply_samples(n: int, lo: int, hi: int, seed: int) -> np.ndarray:
    """n plies drawn uniformly from lo..hi (inclusive): where each sampled
    playout stops to yield a training position."""
    return np.random.default_rng(seed).integers(lo, hi + 1, n).astype(np.int16)
