"""ctypes wrapper for ``ludax_oracle.c`` -- TEST INFRASTRUCTURE ONLY.

Builds ``libludax_oracle.so`` next to the source with plain ``gcc -O2`` (no
intrinsics, no vector pragmas) on first use, then exposes numpy-friendly
functions.  Game ids: 0 Tic-Tac-Toe, 1 Connect Four, 2 Reversi/Othello, 3 Hex,
4 Gomoku, 5 Pente, 6 Yavalath, 7 | L << 8 | flags << 12 the parametric line
game, 8 Wolf and Sheep, 9 English Draughts, 10 Dai Hasami Shogi (move games:
action = from * cells + to; board values 1 / 2 a piece of P1 / P2, 3 / 4 a
Draughts king of P1 / P2; Draughts keeps the cell of a piece that must keep
capturing, plus one, in the passes slot).
Outcome codes: -1 ongoing, 0 draw, 1 P1 win, 2 P2 win, 3 capped.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "ludax_oracle.c")
LIB = os.path.join(HERE, "libludax_oracle.so")

TTT, C4, OTHELLO, HEX, GOMOKU, PENTE, YAVALATH = 0, 1, 2, 3, 4, 5, 6
WOLF_SHEEP, DRAUGHTS, HASAMI_SHOGI = 8, 9, 10    # move games: action = from * cells + to
ONGOING, DRAW, P1, P2, CAPPED = -1, 0, 1, 2, 3

_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle into a shared library (plain scalar C, -O2)."""
    if force or not os.path.exists(LIB) or os.path.getmtime(LIB) < os.path.getmtime(SRC):
        tmp = LIB + f".{os.getpid()}.tmp"
        subprocess.check_call(["gcc", "-O2", "-std=c99", "-fPIC", "-shared", "-o", tmp, SRC, "-lm"])
        os.replace(tmp, LIB)
    return LIB


def lib():
    global _lib
    if _lib is None:
        build()
        L = ctypes.CDLL(LIB)
        u64, i64, i32, u32 = ctypes.c_uint64, ctypes.c_int64, ctypes.c_int32, ctypes.c_uint32
        vp = ctypes.c_void_p
        L.oracle_sm.restype = u64
        L.oracle_sm.argtypes = [u64]
        L.oracle_draw.restype = u64
        L.oracle_draw.argtypes = [u64, u64, u64]
        L.oracle_pick.restype = u32
        L.oracle_pick.argtypes = [u64, u32]
        L.oracle_num_actions.argtypes = [i32, i32, i32]
        L.oracle_num_cells.argtypes = [i32, i32, i32]
        L.oracle_ply_cap.argtypes = [i32, i32, i32]
        L.oracle_hex_connections.argtypes = [i32, vp]
        L.oracle_rollout_start.argtypes = [i32, i32, i32, i64, i64, u64, vp, vp, vp]
        L.oracle_rollout_from.argtypes = [i32, i32, i32, i64, i64, u64, vp, vp, vp, vp, vp, vp]
        L.oracle_step_batch.argtypes = [i32, i32, i32, i64, vp, vp, vp, vp, vp, vp, vp, vp, vp]
        L.oracle_legal_batch.argtypes = [i32, i32, i32, i64, vp, vp, vp, vp, vp, vp]
        L.oracle_reset_batch.argtypes = [i32, i32, i32, i64, vp, vp, vp, vp, vp]
        L.oracle_rollout_mixed.argtypes = [vp, i64, i64, u64, vp, vp]
        L.oracle_perft.restype = u64
        L.oracle_perft.argtypes = [i32, i32, i32, i32]
        L.oracle_perft_turns.restype = u64
        L.oracle_perft_turns.argtypes = [i32, i32, i32, i32]
        L.oracle_ttt_enumerate.argtypes = [vp]
        f64 = ctypes.c_double
        L.oracle_mcts_search.argtypes = [i32, i32, i32, i64, i64, u64, i32, f64, vp, vp, vp, vp, vp, vp, vp, vp]
        L.oracle_mcts_play.argtypes = [i32, i32, i32, i64, i64, u64, i32, i32, f64, vp, vp, vp, vp]
        _lib = L
    return _lib


def _p(a):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


def sm(x: int) -> int:
    return lib().oracle_sm(x & (2**64 - 1))


def draw(seed: int, env: int, ply: int) -> int:
    return lib().oracle_draw(seed, env, ply)


def pick(r: int, n: int) -> int:
    return lib().oracle_pick(r, n)


def num_actions(game, rows, cols) -> int:
    return lib().oracle_num_actions(game, rows, cols)


def num_cells(game, rows, cols) -> int:
    return lib().oracle_num_cells(game, rows, cols)


def ply_cap(game, rows, cols) -> int:
    return lib().oracle_ply_cap(game, rows, cols)


def hex_connections(n: int, cells) -> int:
    c = np.ascontiguousarray(cells, dtype=np.int8)
    return lib().oracle_hex_connections(n, _p(c))


class States:
    """A batch of positions in the canonical layout shared with the C-ABI's
    state view: board[n, cells] int8, to_move/passes/outcome int8, ply int16
    (for Pente, passes holds the captured pairs: P1's in the low 4 bits, P2's
    in the high 4 bits)."""

    def __init__(self, game, rows, cols, n):
        self.game, self.rows, self.cols, self.n = game, rows, cols, n
        self.board = np.zeros((n, num_cells(game, rows, cols)), np.int8)
        self.to_move = np.zeros(n, np.int8)
        self.ply = np.zeros(n, np.int16)
        self.passes = np.zeros(n, np.int8)
        self.outcome = np.zeros(n, np.int8)

    def copy(self):
        s = States(self.game, self.rows, self.cols, self.n)
        for k in ("board", "to_move", "ply", "passes", "outcome"):
            setattr(s, k, getattr(self, k).copy())
        return s

    def _args(self):
        return (_p(self.board), _p(self.to_move), _p(self.ply), _p(self.passes), _p(self.outcome))


def reset(game, rows, cols, n) -> States:
    s = States(game, rows, cols, n)
    assert lib().oracle_reset_batch(game, rows, cols, n, *s._args()) == 0
    return s


def legal(s: States) -> np.ndarray:
    A = num_actions(s.game, s.rows, s.cols)
    out = np.zeros((s.n, A), np.uint8)
    assert lib().oracle_legal_batch(s.game, s.rows, s.cols, s.n, *s._args(), _p(out)) == 0
    return out


def step(s: States, actions):
    """Apply actions[n] in place; returns (rewards[n,2] f32, terminated u8, error u8)."""
    a = np.ascontiguousarray(actions, dtype=np.int32)
    rew = np.zeros((s.n, 2), np.float32)
    term = np.zeros(s.n, np.uint8)
    err = np.zeros(s.n, np.uint8)
    assert lib().oracle_step_batch(s.game, s.rows, s.cols, s.n, *s._args(), _p(a), _p(rew), _p(term), _p(err)) == 0
    return rew, term, err


def rollout_start(game, rows, cols, n, seed, env_offset=0, want_boards=False):
    """Uniform-random playouts from the start position.
    Returns (outcome int8[n], plies int16[n], boards int8[n, cells] or None)."""
    out = np.zeros(n, np.int8)
    plies = np.zeros(n, np.int16)
    boards = np.zeros((n, num_cells(game, rows, cols)), np.int8) if want_boards else None
    assert lib().oracle_rollout_start(game, rows, cols, n, env_offset, seed, _p(boards), _p(out), _p(plies)) == 0
    return out, plies, boards


def rollout_from(s: States, seed, env_offset=0, stop_ply=None):
    """Playouts from the given states (updated in place); stop_ply[n] int16
    stops each env once its ply reaches that value."""
    sp = None if stop_ply is None else np.ascontiguousarray(stop_ply, dtype=np.int16)
    assert lib().oracle_rollout_from(s.game, s.rows, s.cols, s.n, env_offset, seed, *s._args(), _p(sp)) == 0
    return s


def rollout_mixed(desc, seed, env_offset=0):
    d = np.ascontiguousarray(desc, dtype=np.int32)
    n = d.shape[0]
    out = np.zeros(n, np.int8)
    plies = np.zeros(n, np.int16)
    assert lib().oracle_rollout_mixed(_p(d), n, env_offset, seed, _p(out), _p(plies)) == 0
    return out, plies


def mcts_search(s: States, seed, iters, c=2 ** 0.5, env_offset=0):
    """One UCT search per state (see the oracle's MCTS section).  Returns
    (action int32[n] (-1 if over), visits uint32[n, A], wins uint32[n, A])
    with the root children's visit counts and half-point rewards by action."""
    A = num_actions(s.game, s.rows, s.cols)
    act = np.zeros(s.n, np.int32)
    vis = np.zeros((s.n, A), np.uint32)
    win = np.zeros((s.n, A), np.uint32)
    assert lib().oracle_mcts_search(s.game, s.rows, s.cols, s.n, env_offset, seed, iters, c, *s._args(), _p(act),
                                    _p(vis), _p(win)) == 0
    return act, vis, win


def mcts_play(game, rows, cols, n, seed, iters_p1, iters_p2, c=2 ** 0.5, env_offset=0):
    """Matches between UCT agents from the start position.  Returns
    (outcome int8, plies int16, agency int16, coverage int16), each [n]:
    agency = turns with more than one legal action, coverage = cells that
    were occupied at some point."""
    out = np.zeros(n, np.int8)
    plies = np.zeros(n, np.int16)
    agency = np.zeros(n, np.int16)
    cov = np.zeros(n, np.int16)
    assert lib().oracle_mcts_play(game, rows, cols, n, env_offset, seed, iters_p1, iters_p2, c, _p(out), _p(plies),
                                  _p(agency), _p(cov)) == 0
    return out, plies, agency, cov


def perft(game, rows, cols, depth) -> int:
    return lib().oracle_perft(game, rows, cols, depth)


def perft_turns(game, rows, cols, depth) -> int:
    """Perft where a continuation by the same player (a Draughts multi-capture)
    stays at the same depth."""
    return lib().oracle_perft_turns(game, rows, cols, depth)


def ttt_enumerate() -> np.ndarray:
    """counts[length, outcome] over every complete Tic-Tac-Toe game
    (outcome 0 draw, 1 X win, 2 O win)."""
    c = np.zeros(30, np.uint64)
    lib().oracle_ttt_enumerate(_p(c))
    return c.reshape(10, 3)
