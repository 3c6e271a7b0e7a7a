"""Python binding of the C-ABI in ``include/ludax.h`` (argument marshalling only).

Every function below has the name of the C entry point it calls, takes torch
tensors where the C call takes device pointers, checks the returned status and
raises ``LudaxError`` on failure.  All game logic runs in ``libludax.so``'s CUDA
kernels; there is no Python or CPU fallback: importing this module fails when
the library cannot be loaded.

``Env`` wraps an env handle with the same calls as methods.
"""
from __future__ import annotations

import ctypes
import os

import torch

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libludax.so")

LUDAX_OK = 0
LUDAX_GAME_TTT, LUDAX_GAME_C4, LUDAX_GAME_OTHELLO, LUDAX_GAME_HEX = 0, 1, 2, 3
LUDAX_GAME_GOMOKU, LUDAX_GAME_PENTE, LUDAX_GAME_YAVALATH, LUDAX_GAME_LINE = 4, 5, 6, 7
LUDAX_LINE_EXACT, LUDAX_LINE_GRAVITY, LUDAX_LINE_MISERE = 1, 2, 4
LUDAX_GAME_WOLF_SHEEP, LUDAX_GAME_DRAUGHTS, LUDAX_GAME_HASAMI_SHOGI = 8, 9, 10
MOVE_GAMES = (LUDAX_GAME_WOLF_SHEEP, LUDAX_GAME_DRAUGHTS, LUDAX_GAME_HASAMI_SHOGI)
LUDAX_OUTCOME_ONGOING, LUDAX_OUTCOME_DRAW, LUDAX_OUTCOME_P1, LUDAX_OUTCOME_P2, LUDAX_OUTCOME_CAPPED = -1, 0, 1, 2, 3
LUDAX_ROLLOUT_FROM_START, LUDAX_ROLLOUT_WRITE_BACK = 1, 2
LUDAX_MCTS_MAX_ITERS = 4096

GAME_IDS = {"ttt": LUDAX_GAME_TTT, "c4": LUDAX_GAME_C4, "othello": LUDAX_GAME_OTHELLO, "hex": LUDAX_GAME_HEX,
            "gomoku": LUDAX_GAME_GOMOKU, "pente": LUDAX_GAME_PENTE, "yavalath": LUDAX_GAME_YAVALATH,
            "line": LUDAX_GAME_LINE, "wolf_sheep": LUDAX_GAME_WOLF_SHEEP, "draughts": LUDAX_GAME_DRAUGHTS,
            "hasami_shogi": LUDAX_GAME_HASAMI_SHOGI}


def LUDAX_DESC(game: int, rows: int, cols: int) -> int:
    return game | (rows << 8) | (cols << 16)


def LUDAX_DESC_LINE(rows: int, cols: int, line: int, flags: int = 0) -> int:
    return LUDAX_GAME_LINE | (rows << 8) | (cols << 16) | (line << 24) | (flags << 28)


class LudaxError(RuntimeError):
    def __init__(self, status: int, where: str):
        self.status = status
        super().__init__(f"{where}: {status_string(status)} ({status})")


class ludax_board_params(ctypes.Structure):
    _fields_ = [("rows", ctypes.c_int32), ("cols", ctypes.c_int32), ("line", ctypes.c_int32),
                ("flags", ctypes.c_int32)]


class ludax_state_view(ctypes.Structure):
    _fields_ = [("board", ctypes.c_void_p), ("to_move", ctypes.c_void_p), ("ply", ctypes.c_void_p),
                ("passes", ctypes.c_void_p), ("outcome", ctypes.c_void_p)]


class ludax_launch_cfg(ctypes.Structure):
    _fields_ = [("block_threads", ctypes.c_int32), ("blocks_per_sm", ctypes.c_int32),
                ("envs_per_thread", ctypes.c_int32), ("hex_nbr_table", ctypes.c_int32),
                ("compact_every", ctypes.c_int32), ("threads_per_env", ctypes.c_int32),
                ("lanes_per_warp", ctypes.c_int32)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}

    def __repr__(self):
        return f"ludax_launch_cfg({self.as_dict()})"


def make_cfg(block_threads=256, blocks_per_sm=0, envs_per_thread=1, hex_nbr_table=0, compact_every=0,
             threads_per_env=1, lanes_per_warp=0):
    return ludax_launch_cfg(block_threads, blocks_per_sm, envs_per_thread, hex_nbr_table, compact_every,
                            threads_per_env, lanes_per_warp)


_lib = None


def lib() -> ctypes.CDLL:
    """Load libludax.so (raises if it is missing: there is no fallback)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"{LIB_PATH} not found: build it with `python -m paper_2506_22609_b300.build`")
    L = ctypes.CDLL(LIB_PATH)
    i32, i64, u32, u64, vp = ctypes.c_int32, ctypes.c_int64, ctypes.c_uint32, ctypes.c_uint64, ctypes.c_void_p
    P = ctypes.POINTER
    sig = {
        "ludax_env_create": [P(vp), i32, P(ludax_board_params), i64, i64, vp],
        "ludax_env_destroy": [vp],
        "ludax_env_set_stream": [vp, vp],
        "ludax_env_sizes": [vp, P(i32), P(i32), P(i64)],
        "ludax_reset": [vp, vp],
        "ludax_legal_mask": [vp, vp, vp],
        "ludax_step": [vp, vp, vp, vp],
        "ludax_random_step": [vp, u64, vp, vp],
        "ludax_rollout": [vp, u64, u32, vp, vp, vp, P(ludax_launch_cfg)],
        "ludax_rollout_value": [vp, u64, i32, vp, P(ludax_launch_cfg)],
        "ludax_get_state": [vp, P(ludax_state_view)],
        "ludax_set_state": [vp, P(ludax_state_view)],
        "ludax_state_bits_words": [vp, P(i32)],
        "ludax_rollout_host": [vp, vp, vp, u64, vp, vp, P(ludax_launch_cfg)],
        "ludax_rollout_host_packed": [vp, vp, vp, u64, P(ludax_launch_cfg)],
        "ludax_get_state_bits": [vp, vp, vp],
        "ludax_set_state_bits": [vp, vp, vp],
        "ludax_counters": [vp, P(i64), P(i64)],
        "ludax_sync": [vp, i64],
        "ludax_rollout_mixed": [vp, i64, i64, u64, vp, vp, P(ludax_launch_cfg), vp],
        "ludax_mixed_plan_create": [P(vp), vp, i64, i64, P(ludax_launch_cfg), vp, P(i64)],
        "ludax_rollout_mixed_noalloc": [vp, i64, i64, u64, vp, vp, P(ludax_launch_cfg), vp, P(i64)],
        "ludax_mixed_plan_launch": [vp, u64, vp, vp],
        "ludax_mixed_plan_launch_host": [vp, u64, vp, vp, vp],
        "ludax_mixed_plan_sync": [vp, P(i64)],
        "ludax_mixed_plan_destroy": [vp],
        "ludax_autotune": [vp, i64, u64, i32, vp, P(ludax_launch_cfg), P(ctypes.c_float), vp, P(i32)],
        "ludax_autotune_env": [vp, u64, i32, P(ludax_launch_cfg), P(ctypes.c_float), vp, P(i32)],
        "ludax_autotune_candidates": [P(ludax_launch_cfg), i32],
        "ludax_autotune_env_candidates": [vp, P(ludax_launch_cfg), i32],
        "ludax_net_create": [P(vp), i32, i64, vp],
        "ludax_net_destroy": [vp],
        "ludax_net_sizes": [vp, P(i32), P(i32), P(i64)],
        "ludax_net_set_params": [vp, vp],
        "ludax_net_get_params": [vp, vp],
        "ludax_net_get_state": [vp, vp, vp, vp, P(i64)],
        "ludax_net_set_state": [vp, vp, vp, vp, i64],
        "ludax_net_set_tensor_path": [vp, i32],
        "ludax_net_forward": [vp, vp, i64, vp],
        "ludax_net_grad": [vp, vp, vp, i64, vp, vp],
        "ludax_net_train_step": [vp, vp, vp, i64, ctypes.c_float, vp],
        "ludax_pack_inputs": [vp, vp, i32],
        "ludax_truncated_value": [vp, vp, u64, i32, i32, vp],
        "ludax_dense_bf16_relu": [vp, vp, vp, vp, i32, i32, i32, i32, vp],
        "ludax_device_error": [P(i32)],
        "ludax_int_peak": [i32, i64, P(i64), vp],
        "ludax_selftest_wait": [i64, vp],
        "ludax_mcts_reserve": [vp, i32, ctypes.c_double],
        "ludax_mcts_search": [vp, u64, i32, ctypes.c_double, vp, vp, vp],
        "ludax_mcts_play": [vp, u64, u32, i32, i32, ctypes.c_double, vp, vp, vp, vp],
        "ludax_mcts_play_mixed": [vp, vp, i64, i64, u64, ctypes.c_double, vp, vp, vp, vp, vp, P(i64)],
    }
    for name, args in sig.items():
        fn = getattr(L, name)
        fn.argtypes = args
        fn.restype = ctypes.c_int
    L.ludax_status_string.argtypes = [ctypes.c_int]
    L.ludax_status_string.restype = ctypes.c_char_p
    _lib = L
    return L


def status_string(status: int) -> str:
    return lib().ludax_status_string(status).decode()


def _check(status: int, where: str):
    if status != LUDAX_OK:
        raise LudaxError(status, where)


def _ptr(t):
    if t is None:
        return None
    if not isinstance(t, torch.Tensor):
        raise TypeError("expected a torch tensor")
    if not t.is_cuda:
        raise ValueError("expected a CUDA tensor (device memory)")
    if not t.is_contiguous():
        raise ValueError("expected a contiguous tensor")
    return ctypes.c_void_p(t.data_ptr())


def _stream(stream):
    if stream is None:
        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(stream.cuda_stream)


# ------------------------------------------------------------- C-ABI calls --
def ludax_env_create(game: int, rows: int, cols: int, num_envs: int, env_offset: int = 0, stream=None, line: int = 0,
                     flags: int = 0):
    h = ctypes.c_void_p()
    p = ludax_board_params(rows, cols, line, flags)
    _check(lib().ludax_env_create(ctypes.byref(h), game, ctypes.byref(p), num_envs, env_offset, _stream(stream)),
           "ludax_env_create")
    return h


def ludax_env_destroy(h):
    _check(lib().ludax_env_destroy(h), "ludax_env_destroy")


def ludax_env_set_stream(h, stream):
    _check(lib().ludax_env_set_stream(h, _stream(stream)), "ludax_env_set_stream")


def ludax_env_sizes(h):
    a, w, n = ctypes.c_int32(), ctypes.c_int32(), ctypes.c_int64()
    _check(lib().ludax_env_sizes(h, ctypes.byref(a), ctypes.byref(w), ctypes.byref(n)), "ludax_env_sizes")
    return a.value, w.value, n.value


def ludax_reset(h, env_mask=None):
    _check(lib().ludax_reset(h, _ptr(env_mask)), "ludax_reset")


def ludax_legal_mask(h, mask, pass_legal=None):
    _check(lib().ludax_legal_mask(h, _ptr(mask), _ptr(pass_legal)), "ludax_legal_mask")


def ludax_step(h, actions, rewards, terminated):
    _check(lib().ludax_step(h, _ptr(actions), _ptr(rewards), _ptr(terminated)), "ludax_step")


def ludax_random_step(h, seed: int, rewards, terminated):
    _check(lib().ludax_random_step(h, seed, _ptr(rewards), _ptr(terminated)), "ludax_random_step")


def ludax_rollout(h, seed: int, flags: int, stop_ply=None, outcome=None, plies=None, cfg=None):
    _check(lib().ludax_rollout(h, seed, flags, _ptr(stop_ply), _ptr(outcome), _ptr(plies),
                               ctypes.byref(cfg) if cfg is not None else None), "ludax_rollout")


def ludax_rollout_value(h, seed: int, R: int, value, cfg=None):
    _check(lib().ludax_rollout_value(h, seed, R, _ptr(value), ctypes.byref(cfg) if cfg is not None else None),
           "ludax_rollout_value")


def _view(board, to_move, ply, passes, outcome):
    return ludax_state_view(*(t.data_ptr() for t in (board, to_move, ply, passes, outcome)))


def ludax_get_state(h, board, to_move, ply, passes, outcome):
    for t in (board, to_move, ply, passes, outcome):
        _ptr(t)
    v = _view(board, to_move, ply, passes, outcome)
    _check(lib().ludax_get_state(h, ctypes.byref(v)), "ludax_get_state")


def ludax_set_state(h, board, to_move, ply, passes, outcome):
    for t in (board, to_move, ply, passes, outcome):
        _ptr(t)
    v = _view(board, to_move, ply, passes, outcome)
    _check(lib().ludax_set_state(h, ctypes.byref(v)), "ludax_set_state")


def ludax_state_bits_words(h) -> int:
    w = ctypes.c_int32()
    _check(lib().ludax_state_bits_words(h, ctypes.byref(w)), "ludax_state_bits_words")
    return w.value


def ludax_get_state_bits(h, planes, meta):
    """planes int64 [words_per_env][n] (uint64 bits), meta int32 [n] (uint32 bits)."""
    _check(lib().ludax_get_state_bits(h, _ptr(planes), _ptr(meta)), "ludax_get_state_bits")


def ludax_set_state_bits(h, planes, meta):
    _check(lib().ludax_set_state_bits(h, _ptr(planes), _ptr(meta)), "ludax_set_state_bits")


def ludax_rollout_host(h, planes_host, meta_host, seed, outcome_host, plies_host, cfg=None):
    """Host tensors (pinned for asynchronous copies): planes int64
    [words_per_env][n], meta int32 [n] in; outcome int8 [n], plies int16 [n]
    out, valid once the env's stream has reached this call."""
    for t in (planes_host, meta_host, outcome_host, plies_host):
        if t.is_cuda or not t.is_contiguous():
            raise ValueError("ludax_rollout_host takes contiguous host tensors")
    _check(lib().ludax_rollout_host(h, planes_host.data_ptr(), meta_host.data_ptr(), seed, outcome_host.data_ptr(),
                                    plies_host.data_ptr(), ctypes.byref(cfg) if cfg is not None else None),
           "ludax_rollout_host")


def ludax_rollout_host_packed(h, in_host, out_host, seed, cfg=None):
    """in_host uint8 host tensor: planes then meta; out_host uint8: outcome,
    a pad byte when n is odd, then plies."""
    for t in (in_host, out_host):
        if t.is_cuda or not t.is_contiguous():
            raise ValueError("ludax_rollout_host_packed takes contiguous host tensors")
    _check(lib().ludax_rollout_host_packed(h, in_host.data_ptr(), out_host.data_ptr(), seed,
                                           ctypes.byref(cfg) if cfg is not None else None),
           "ludax_rollout_host_packed")


def ludax_counters(h):
    a, b = ctypes.c_int64(), ctypes.c_int64()
    _check(lib().ludax_counters(h, ctypes.byref(a), ctypes.byref(b)), "ludax_counters")
    return a.value, b.value


def ludax_sync(h, timeout_ms: int = -1):
    _check(lib().ludax_sync(h, timeout_ms), "ludax_sync")


def ludax_rollout_mixed(desc, env_offset: int, seed: int, outcome, plies, cfg=None, stream=None):
    _check(lib().ludax_rollout_mixed(_ptr(desc), desc.numel(), env_offset, seed, _ptr(outcome), _ptr(plies),
                                     ctypes.byref(cfg) if cfg is not None else None, _stream(stream)),
           "ludax_rollout_mixed")


def ludax_rollout_mixed_noalloc(desc, env_offset: int, seed: int, outcome, plies, cfg=None, stream=None):
    """Allocation-free mixed-batch playout (at most 2^20 envs; calls share one
    static scratch array and must not overlap on the GPU)."""
    bad = ctypes.c_int64(-1)
    st = lib().ludax_rollout_mixed_noalloc(_ptr(desc), desc.numel(), env_offset, seed, _ptr(outcome), _ptr(plies),
                                           ctypes.byref(cfg) if cfg is not None else None, _stream(stream),
                                           ctypes.byref(bad))
    if st != LUDAX_OK:
        err = LudaxError(st, f"ludax_rollout_mixed_noalloc (first bad descriptor index {bad.value})")
        err.bad_index = bad.value
        raise err


def ludax_mcts_reserve(h, iterations: int, c: float):
    _check(lib().ludax_mcts_reserve(h, iterations, c), "ludax_mcts_reserve")


def ludax_mcts_search(h, seed: int, iterations: int, c: float, action, visits=None, wins=None):
    _check(lib().ludax_mcts_search(h, seed, iterations, c, _ptr(action), _ptr(visits), _ptr(wins)),
           "ludax_mcts_search")


def ludax_mcts_play(h, seed: int, flags: int, iters_p1: int, iters_p2: int, c: float, outcome=None, plies=None,
                    agency=None, coverage=None):
    _check(lib().ludax_mcts_play(h, seed, flags, iters_p1, iters_p2, c, _ptr(outcome), _ptr(plies), _ptr(agency),
                                 _ptr(coverage)), "ludax_mcts_play")


def ludax_mcts_play_mixed(desc, iters, env_offset: int, seed: int, c: float, outcome=None, plies=None, agency=None,
                          coverage=None, stream=None):
    """desc: host int32 [n] descriptors; iters: host int32 [n, 2] (P1, P2)."""
    import numpy as np

    d = np.ascontiguousarray(desc, dtype=np.int32)
    it = np.ascontiguousarray(iters, dtype=np.int32)
    if it.shape != (d.shape[0], 2):
        raise ValueError("iters must have shape [n, 2]")
    bad = ctypes.c_int64(-1)
    st = lib().ludax_mcts_play_mixed(d.ctypes.data_as(ctypes.c_void_p), it.ctypes.data_as(ctypes.c_void_p), d.shape[0],
                                     env_offset, seed, c, _ptr(outcome), _ptr(plies), _ptr(agency), _ptr(coverage),
                                     _stream(stream), ctypes.byref(bad))
    if st != LUDAX_OK:
        err = LudaxError(st, f"ludax_mcts_play_mixed (first bad index {bad.value})")
        err.bad_index = bad.value
        raise err


def ludax_mixed_plan_create(desc, env_offset: int = 0, cfg=None, stream=None):
    h = ctypes.c_void_p()
    bad = ctypes.c_int64(-1)
    st = lib().ludax_mixed_plan_create(ctypes.byref(h), _ptr(desc), desc.numel(), env_offset,
                                       ctypes.byref(cfg) if cfg is not None else None, _stream(stream),
                                       ctypes.byref(bad))
    if st != LUDAX_OK:
        err = LudaxError(st, f"ludax_mixed_plan_create (first bad descriptor index {bad.value})")
        err.bad_index = bad.value
        raise err
    return h


def ludax_mixed_plan_launch(plan, seed: int, outcome, plies):
    _check(lib().ludax_mixed_plan_launch(plan, seed, _ptr(outcome), _ptr(plies)), "ludax_mixed_plan_launch")


def ludax_mixed_plan_launch_host(plan, seed: int, desc_host, outcome_host, plies_host):
    """Host tensors (pinned for asynchronous copies): desc int32 [n] in,
    outcome int8 [n] and plies int16 [n] out, valid once the plan's stream
    has reached this call (ludax_mixed_plan_sync)."""
    for t in (desc_host, outcome_host, plies_host):
        if t.is_cuda or not t.is_contiguous():
            raise ValueError("ludax_mixed_plan_launch_host takes contiguous host tensors")
    _check(lib().ludax_mixed_plan_launch_host(plan, seed, desc_host.data_ptr(), outcome_host.data_ptr(),
                                              plies_host.data_ptr()), "ludax_mixed_plan_launch_host")


def ludax_mixed_plan_sync(plan):
    bad = ctypes.c_int64(-1)
    st = lib().ludax_mixed_plan_sync(plan, ctypes.byref(bad))
    if st != 0:
        err = LudaxError(st, f"ludax_mixed_plan_sync (first bad descriptor index {bad.value})")
        err.bad_index = bad.value
        raise err


def ludax_mixed_plan_destroy(plan):
    _check(lib().ludax_mixed_plan_destroy(plan), "ludax_mixed_plan_destroy")


def ludax_autotune_candidates():
    n = lib().ludax_autotune_candidates(None, 0)
    arr = (ludax_launch_cfg * n)()
    lib().ludax_autotune_candidates(arr, n)
    return list(arr)


def ludax_autotune(desc, seed: int = 0, reps: int = 5, stream=None):
    """Returns (best cfg, best median ms, [(cfg, ms) per candidate])."""
    cands = ludax_autotune_candidates()
    best = ludax_launch_cfg()
    best_ms = ctypes.c_float()
    table = (ctypes.c_float * len(cands))()
    nc = ctypes.c_int32()
    _check(lib().ludax_autotune(_ptr(desc), desc.numel(), seed, reps, _stream(stream), ctypes.byref(best),
                                ctypes.byref(best_ms), table, ctypes.byref(nc)), "ludax_autotune")
    return best, best_ms.value, list(zip(cands, list(table)))


def ludax_autotune_env_candidates(h):
    n = lib().ludax_autotune_env_candidates(h, None, 0)
    arr = (ludax_launch_cfg * n)()
    lib().ludax_autotune_env_candidates(h, arr, n)
    return list(arr)


def ludax_autotune_env(h, seed: int = 0, reps: int = 5):
    """Autotunes ludax_rollout (from the start position) for one env batch:
    (best config, its median ms, [(candidate, median ms), ...])."""
    cands_n = ctypes.c_int32()
    best = ludax_launch_cfg()
    best_ms = ctypes.c_float()
    table = (ctypes.c_float * 512)()
    _check(lib().ludax_autotune_env(h, seed, reps, ctypes.byref(best), ctypes.byref(best_ms), table,
                                    ctypes.byref(cands_n)), "ludax_autotune_env")
    return best, best_ms.value, list(zip(ludax_autotune_env_candidates(h), list(table)[: cands_n.value]))


def ludax_net_create(cells: int, max_batch: int, stream=None):
    h = ctypes.c_void_p()
    _check(lib().ludax_net_create(ctypes.byref(h), cells, max_batch, _stream(stream)), "ludax_net_create")
    return h


def ludax_net_destroy(h):
    _check(lib().ludax_net_destroy(h), "ludax_net_destroy")


def ludax_net_sizes(h):
    a, b, c = ctypes.c_int32(), ctypes.c_int32(), ctypes.c_int64()
    _check(lib().ludax_net_sizes(h, ctypes.byref(a), ctypes.byref(b), ctypes.byref(c)), "ludax_net_sizes")
    return a.value, b.value, c.value


def ludax_net_set_params(h, params):
    _check(lib().ludax_net_set_params(h, _ptr(params)), "ludax_net_set_params")


def ludax_net_get_params(h, params):
    _check(lib().ludax_net_get_params(h, _ptr(params)), "ludax_net_get_params")


def ludax_net_get_state(h, params, m, v):
    """Copies parameters and Adam's moments into the three device tensors;
    returns the number of Adam steps taken."""
    steps = ctypes.c_int64()
    _check(lib().ludax_net_get_state(h, _ptr(params), _ptr(m), _ptr(v), ctypes.byref(steps)), "ludax_net_get_state")
    return steps.value


def ludax_net_set_state(h, params, m, v, steps):
    _check(lib().ludax_net_set_state(h, _ptr(params), _ptr(m), _ptr(v), int(steps)), "ludax_net_set_state")


def ludax_net_forward(h, x, p):
    _check(lib().ludax_net_forward(h, _ptr(x), x.shape[0], _ptr(p)), "ludax_net_forward")


def ludax_net_grad(h, x, y, grad=None, loss=None):
    _check(lib().ludax_net_grad(h, _ptr(x), _ptr(y), x.shape[0], _ptr(grad), _ptr(loss)), "ludax_net_grad")


def ludax_net_train_step(h, x, y, lr: float, loss=None):
    _check(lib().ludax_net_train_step(h, _ptr(x), _ptr(y), x.shape[0], lr, _ptr(loss)), "ludax_net_train_step")


def ludax_pack_inputs(env_h, x, ld: int):
    _check(lib().ludax_pack_inputs(env_h, _ptr(x), ld), "ludax_pack_inputs")


def ludax_truncated_value(env_h, net_h, seed: int, K: int, plies: int, value):
    _check(lib().ludax_truncated_value(env_h, net_h, seed, K, plies, _ptr(value)), "ludax_truncated_value")


def ludax_dense_bf16_relu(a, b, bias, out, stream=None):
    M, K = a.shape
    N = b.shape[0]
    _check(lib().ludax_dense_bf16_relu(_ptr(a), _ptr(b), _ptr(bias), _ptr(out), M, N, K, out.shape[1],
                                       _stream(stream)), "ludax_dense_bf16_relu")


def ludax_device_error():
    e = ctypes.c_int32()
    lib().ludax_device_error(ctypes.byref(e))
    return e.value


def ludax_selftest_wait(limit_cycles: int, stream=None):
    """Make a bounded device wait expire (see ludax_device_error)."""
    _check(lib().ludax_selftest_wait(limit_cycles, _stream(stream)), "ludax_selftest_wait")


INT_PEAK_KINDS = {"lop3": 0, "iadd": 1, "shf": 2, "imad": 3, "imad_hi": 4, "lop3_imad": 5}


def ludax_int_peak(kind: str, iters: int, stream=None) -> int:
    """Launch the integer-issue microbenchmark; returns the number of ops."""
    ops = ctypes.c_int64()
    _check(lib().ludax_int_peak(INT_PEAK_KINDS[kind], iters, ctypes.byref(ops), _stream(stream)), "ludax_int_peak")
    return ops.value


class Net:
    """The value network (bf16 inputs are passed as int16 tensors holding the bits)."""

    def __init__(self, cells, max_batch, stream=None):
        self.handle = ludax_net_create(cells, max_batch, stream)
        self.in_pad, self.hidden, self.num_params = ludax_net_sizes(self.handle)
        self.cells, self.max_batch = cells, max_batch

    def close(self):
        if getattr(self, "handle", None) is not None:
            ludax_net_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_params(self, params):
        ludax_net_set_params(self.handle, params.to(torch.float32).contiguous())

    def set_tensor_path(self, use_tcgen05):
        """True / 1: tcgen05 (one-launch MLP for inference; tcgen05 backward),
        2: tcgen05 as two layer launches, False / 0: mma.sync everywhere."""
        mode = int(use_tcgen05) if not isinstance(use_tcgen05, bool) else (1 if use_tcgen05 else 0)
        _check(lib().ludax_net_set_tensor_path(self.handle, mode), "ludax_net_set_tensor_path")

    def get_params(self):
        p = torch.empty(self.num_params, dtype=torch.float32, device="cuda")
        ludax_net_get_params(self.handle, p)
        return p

    def get_state(self):
        """(parameters, Adam m, Adam v, Adam steps taken): what set_state needs
        to continue training exactly where this net stands."""
        p, m, v = (torch.empty(self.num_params, dtype=torch.float32, device="cuda") for _ in range(3))
        steps = ludax_net_get_state(self.handle, p, m, v)
        return p, m, v, steps

    def set_state(self, params, m, v, steps):
        f = lambda t: t.to(device="cuda", dtype=torch.float32).contiguous()  # noqa: E731
        ludax_net_set_state(self.handle, f(params), f(m), f(v), steps)

    def forward(self, x):
        p = torch.empty(x.shape[0], dtype=torch.float32, device="cuda")
        ludax_net_forward(self.handle, x, p)
        return p

    def grad(self, x, y):
        g = torch.empty(self.num_params, dtype=torch.float32, device="cuda")
        loss = torch.empty(1, dtype=torch.float32, device="cuda")
        ludax_net_grad(self.handle, x, y, g, loss)
        return g, loss

    def train_step(self, x, y, lr):
        loss = torch.empty(1, dtype=torch.float32, device="cuda")
        ludax_net_train_step(self.handle, x, y, lr, loss)
        return loss


# ------------------------------------------------------------------- Env ----
class Env:
    """A batch of num_envs envs of one game on the current CUDA device."""

    def __init__(self, game, rows, cols, num_envs, env_offset=0, stream=None, device=None, line=0, flags=0):
        if isinstance(game, str):
            game = GAME_IDS[game]
        self.device = torch.device(device) if device is not None else torch.device("cuda", torch.cuda.current_device())
        self.game, self.rows, self.cols, self.num_envs, self.env_offset = game, rows, cols, num_envs, env_offset
        self.stream = stream
        with torch.cuda.device(self.device):
            self.handle = ludax_env_create(game, rows, cols, num_envs, env_offset, stream, line, flags)
        self.num_actions, self.mask_words, _ = ludax_env_sizes(self.handle)
        if game in MOVE_GAMES:  # action = from * cells + to
            self.cells = int(round(self.num_actions ** 0.5))
        else:
            self.cells = self.num_actions - (1 if game == LUDAX_GAME_OTHELLO else 0)

    def close(self):
        if getattr(self, "handle", None) is not None:
            ludax_env_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _empty(self, shape, dtype):
        return torch.empty(shape, dtype=dtype, device=self.device)

    def reset(self, env_mask=None):
        ludax_reset(self.handle, env_mask)

    def legal_mask(self):
        m = self._empty((self.num_envs, self.mask_words), torch.int64)
        p = self._empty((self.num_envs,), torch.uint8)
        ludax_legal_mask(self.handle, m, p)
        return m, p

    def step(self, actions):
        r = self._empty((self.num_envs, 2), torch.float32)
        t = self._empty((self.num_envs,), torch.uint8)
        ludax_step(self.handle, actions.to(torch.int32).contiguous(), r, t)
        return r, t

    def random_step(self, seed):
        r = self._empty((self.num_envs, 2), torch.float32)
        t = self._empty((self.num_envs,), torch.uint8)
        ludax_random_step(self.handle, seed, r, t)
        return r, t

    def rollout(self, seed, from_start=True, write_back=False, stop_ply=None, cfg=None, outcome=None, plies=None):
        flags = (LUDAX_ROLLOUT_FROM_START if from_start else 0) | (LUDAX_ROLLOUT_WRITE_BACK if write_back else 0)
        out = outcome if outcome is not None else self._empty((self.num_envs,), torch.int8)
        pl = plies if plies is not None else self._empty((self.num_envs,), torch.int16)
        ludax_rollout(self.handle, seed, flags, stop_ply, out, pl, cfg)
        return out, pl

    def rollout_value(self, seed, R, cfg=None):
        v = self._empty((self.num_envs,), torch.float32)
        ludax_rollout_value(self.handle, seed, R, v, cfg)
        return v

    def mcts_search(self, seed, iterations, c=2 ** 0.5, stats=False):
        """One UCT search per env from its current state: the chosen action
        ids, and with stats=True the root children's visits and half-point
        rewards by action id."""
        act = self._empty((self.num_envs,), torch.int32)
        vis = self._empty((self.num_envs, self.num_actions), torch.int32) if stats else None
        win = self._empty((self.num_envs, self.num_actions), torch.int32) if stats else None
        ludax_mcts_search(self.handle, seed, iterations, c, act, vis, win)
        return (act, vis, win) if stats else act

    def mcts_reserve(self, iterations, c=2 ** 0.5):
        ludax_mcts_reserve(self.handle, iterations, c)

    def mcts_play(self, seed, iters_p1, iters_p2, c=2 ** 0.5, from_start=True, write_back=False):
        """One match per env between UCT agents: (outcome, plies, agency,
        coverage) per env."""
        flags = (LUDAX_ROLLOUT_FROM_START if from_start else 0) | (LUDAX_ROLLOUT_WRITE_BACK if write_back else 0)
        n = self.num_envs
        out = self._empty((n,), torch.int8)
        pl, ag, cov = (self._empty((n,), torch.int16) for _ in range(3))
        ludax_mcts_play(self.handle, seed, flags, iters_p1, iters_p2, c, out, pl, ag, cov)
        return out, pl, ag, cov

    def get_state(self):
        n = self.num_envs
        board = self._empty((n, self.cells), torch.int8)
        to_move = self._empty((n,), torch.int8)
        ply = self._empty((n,), torch.int16)
        passes = self._empty((n,), torch.int8)
        outcome = self._empty((n,), torch.int8)
        ludax_get_state(self.handle, board, to_move, ply, passes, outcome)
        return board, to_move, ply, passes, outcome

    def set_state(self, board, to_move, ply, passes, outcome):
        ts = [t.to(self.device).contiguous() for t in (board, to_move, ply, passes, outcome)]
        ludax_set_state(self.handle, *ts)
        ludax_sync(self.handle)  # the temporaries in ts must outlive the copy

    def state_bits_words(self):
        return ludax_state_bits_words(self.handle)

    def get_state_bits(self):
        """(planes int64 [words_per_env][n], meta int32 [n]): the packed state."""
        planes = self._empty((self.state_bits_words(), self.num_envs), torch.int64)
        meta = self._empty((self.num_envs,), torch.int32)
        ludax_get_state_bits(self.handle, planes, meta)
        return planes, meta

    def set_state_bits(self, planes, meta):
        ts = [t.to(self.device).contiguous() for t in (planes, meta)]
        ludax_set_state_bits(self.handle, *ts)
        ludax_sync(self.handle)  # the temporaries in ts must outlive the copy

    def counters(self):
        return ludax_counters(self.handle)

    def sync(self, timeout_ms=-1):
        ludax_sync(self.handle, timeout_ms)
