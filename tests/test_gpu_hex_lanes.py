"""GPU: Hex playouts with several lanes per env (threads_per_env 2 and 4)
against the CPU oracle, bit for bit.

The lanes of a group split the board's words and share the draw, the k-th
legal cell and the end tests through shuffles; the results must not depend
on that split: outcomes, game lengths and final boards equal the oracle's on
every board size 2..11, from the start position and from stored positions,
with stop plies and write-back, in persistent (refilling) and one-group-per-
env launch shapes, with and without the shared-memory neighbour table.
"""
import numpy as np
import pytest
import torch

from oracle import games as G
from paper_2506_22609_b300 import workloads as W

pytestmark = pytest.mark.gpu

SHAPES = [(256, 0, 1, 0, 0, 2), (64, 1, 1, 1, 0, 2), (128, 0, 1, 1, 0, 4), (96, 2, 1, 0, 0, 4),
          (512, 3, 1, 1, 0, 2), (32, 1, 1, 0, 0, 4)]


def np_(t):
    return t.detach().cpu().numpy()


@pytest.mark.parametrize("cfg", SHAPES, ids=lambda c: "b{}_bps{}_tab{}_tpe{}".format(c[0], c[1], c[3], c[5]))
@pytest.mark.parametrize("size", [2, 3, 4, 5, 7, 8, 9, 11])
def test_lanes_from_start_match_oracle(L, size, cfg):
    n, seed, off = 2600, 5, 911
    env = L.Env("hex", size, size, n, env_offset=off)
    out, plies = env.rollout(seed, from_start=True, write_back=True, cfg=L.make_cfg(*cfg))
    o_out, o_plies, o_boards = G.rollout_start(G.HEX, size, size, n, seed, env_offset=off, want_boards=True)
    assert (np_(out) == o_out).all() and (np_(plies) == o_plies).all()
    b, tm, ply, ps, oc = env.get_state()
    assert (np_(b) == o_boards).all() and (np_(oc) == o_out).all() and (np_(ply) == o_plies).all()
    assert env.counters() == (0, 0)  # nothing capped, nothing illegal
    env.close()


@pytest.mark.parametrize("tpe", [2, 4])
@pytest.mark.parametrize("size", [5, 9, 11])
def test_lanes_from_stored_positions_with_stop_plies(L, size, tpe):
    n = 1500
    rng = np.random.default_rng(size * 7 + tpe)
    s = G.reset(G.HEX, size, size, n)
    G.rollout_from(s, seed=3, stop_ply=rng.integers(0, size * size, n).astype(np.int16))
    env = L.Env("hex", size, size, n, env_offset=40)
    env.set_state(*(torch.from_numpy(x) for x in (s.board, s.to_move, s.ply, s.passes, s.outcome)))
    cfg = L.make_cfg(128, 1, 1, 1, 0, tpe)
    # a partial playout to stop plies, written back, then the rest of the game
    stop = (s.ply + rng.integers(0, 9, n)).astype(np.int16)
    s2 = s.copy()
    G.rollout_from(s2, seed=9, env_offset=40, stop_ply=stop)
    out, plies = env.rollout(9, from_start=False, write_back=True, stop_ply=torch.from_numpy(stop).cuda(), cfg=cfg)
    b, tm, ply, ps, oc = env.get_state()
    assert (np_(b) == s2.board).all() and (np_(tm) == s2.to_move).all() and (np_(ply) == s2.ply).all()
    assert (np_(oc) == s2.outcome).all()
    assert (np_(out) == s2.outcome).all() and (np_(plies) == s2.ply).all()
    # the written-back edge sets are exact: the rest of the game, with lanes or with one lane per env
    G.rollout_from(s2, seed=10, env_offset=40)
    out, plies = env.rollout(10, from_start=False, write_back=True, cfg=cfg if tpe == 4 else None)
    b, tm, ply, ps, oc = env.get_state()
    assert (np_(b) == s2.board).all() and (np_(oc) == s2.outcome).all() and (np_(ply) == s2.ply).all()
    env.close()


@pytest.mark.parametrize("n", [1, 31, 33, 257])
def test_lanes_ragged_batches(L, n):
    for size in (7, 11):
        env = L.Env("hex", size, size, n)
        o, p, _ = G.rollout_start(G.HEX, size, size, n, 11)
        for cfg in [(64, 1, 1, 0, 0, 2), (32, 1, 1, 1, 0, 4), (256, 0, 1, 1, 0, 4)]:
            out, plies = env.rollout(11, cfg=L.make_cfg(*cfg))
            assert (np_(out) == o).all() and (np_(plies) == p).all()
        env.close()


def test_lanes_benchmark_size_sampled(L):
    cfg = W.HEX11_64K
    env = L.Env("hex", 11, 11, cfg.num_envs)
    for shape in [(256, 0, 1, 1, 0, 2), (256, 0, 1, 1, 0, 4), (448, 2, 1, 1, 0, 2)]:
        out, plies = env.rollout(cfg.seed, cfg=L.make_cfg(*shape))
        ref_out, ref_plies = env.rollout(cfg.seed, cfg=L.make_cfg(*W.bench_cfg(cfg)))
        assert torch.equal(out, ref_out) and torch.equal(plies, ref_plies)
    out, plies = np_(out), np_(plies)
    for e in W.sample_envs(cfg.num_envs, 300, 2):
        o, p, _ = G.rollout_start(G.HEX, 11, 11, 1, cfg.seed, env_offset=int(e))
        assert o[0] == out[e] and p[0] == plies[e]
    env.close()


def test_lanes_argument_checks(L):
    env = L.Env("c4", 6, 7, 64)
    with pytest.raises(L.LudaxError) as ei:  # several lanes per env: Hex only
        env.rollout(1, cfg=L.make_cfg(64, 0, 1, 0, 0, 2))
    assert ei.value.status == -1
    env.close()
    env = L.Env("hex", 5, 5, 64)
    for bad in [(64, 0, 1, 0, 0, 3), (64, 0, 2, 0, 0, 2), (64, 0, 1, 0, 4, 2), (64, 0, 1, 0, 0, 8)]:
        with pytest.raises(L.LudaxError) as ei:
            env.rollout(1, cfg=L.make_cfg(*bad))
        assert ei.value.status == -1
    with pytest.raises(L.LudaxError):  # the value playouts run one lane per env
        env.rollout_value(1, 4, cfg=L.make_cfg(64, 0, 1, 0, 0, 2))
    env.close()


def test_env_autotuner_walks_lanes_per_env(L):
    env = L.Env("hex", 9, 9, 4096)
    cands = L.ludax_autotune_env_candidates(env.handle)
    assert {c.threads_per_env for c in cands} == {1, 2, 4}
    assert {c.lanes_per_warp for c in cands} == {0, 8, 16}  # part-filled warps (one lane per env)
    best, best_ms, table = L.ludax_autotune_env(env.handle, 1, reps=1)
    assert len(table) == len(cands) and best_ms == min(ms for _, ms in table)
    env.close()
