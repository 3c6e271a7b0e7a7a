"""Move games on the GPU (App. C: Wolf and Sheep, English Draughts, Dai
Hasami Shogi; action = from * cells + to) against the oracle, element by
element: playouts, legal masks and steps along oracle-driven games, state
round trips, partial playouts, mixed batches, UCT searches and matches."""
import numpy as np
import pytest
import torch

from oracle import games as G
from paper_2506_22609_b300 import workloads as W

pytestmark = pytest.mark.gpu

MOVE = [("wolf_sheep", G.WOLF_SHEEP, 8, 8, 4000), ("draughts", G.DRAUGHTS, 8, 8, 3000),
        ("hasami_shogi", G.HASAMI_SHOGI, 9, 9, 800)]


def np_(t):
    return t.detach().cpu().numpy()


def push(env, s):
    env.set_state(*(torch.from_numpy(x) for x in (s.board, s.to_move, s.ply, s.passes, s.outcome)))


def assert_same_state(env, s):
    b, tm, ply, ps, oc = env.get_state()
    torch.cuda.synchronize()
    assert (np_(b) == s.board).all()
    assert (np_(tm) == s.to_move).all() and (np_(ply) == s.ply).all()
    assert (np_(ps) == s.passes).all() and (np_(oc) == s.outcome).all()


@pytest.mark.parametrize("name,game,rows,cols,n", MOVE, ids=[m[0] for m in MOVE])
def test_playouts_match_oracle(L, name, game, rows, cols, n):
    env = L.Env(game, rows, cols, n, env_offset=9)
    assert env.num_actions == (rows * cols) ** 2 and env.cells == rows * cols
    out, plies = env.rollout(17, write_back=True)
    o, p, b = G.rollout_start(game, rows, cols, n, 17, env_offset=9, want_boards=True)
    assert (np_(out) == o).all() and (np_(plies) == p).all()
    board, *_ = env.get_state()
    torch.cuda.synchronize()
    assert (np_(board) == b).all()
    env.close()


@pytest.mark.parametrize("name,game,rows,cols,n", MOVE, ids=[m[0] for m in MOVE])
def test_launch_shapes_agree(L, name, game, rows, cols, n):
    env = L.Env(game, rows, cols, n)
    ref = [np_(t) for t in env.rollout(3)]
    for cfg in (L.make_cfg(128, 2, 1, 0, 0), L.make_cfg(256, 4, 2, 0, 0), L.make_cfg(448, 4, 1, 0, 8)):
        got = [np_(t) for t in env.rollout(3, cfg=cfg)]
        assert all((a == b).all() for a, b in zip(ref, got))
    env.close()


@pytest.mark.parametrize("name,game,rows,cols,n", MOVE, ids=[m[0] for m in MOVE])
def test_step_api_along_oracle_games(L, name, game, rows, cols, n):
    m = 64
    A = (rows * cols) ** 2
    env = L.Env(game, rows, cols, m)
    s = G.reset(game, rows, cols, m)
    rng = np.random.default_rng(rows + game)
    for _ in range(200):
        legal = G.legal(s)
        mk, _pass = env.legal_mask()
        torch.cuda.synchronize()
        bits = np.unpackbits(np_(mk).view(np.uint8), axis=1, bitorder="little")[:, :A]
        assert (bits == legal).all()
        acts = np.array([rng.choice(np.flatnonzero(lg)) if lg.any() else 0 for lg in legal], np.int32)
        o_rew, o_term, _ = G.step(s, acts)
        rew, term = env.step(torch.from_numpy(acts).cuda())
        torch.cuda.synchronize()
        assert (np_(rew) == o_rew).all() and (np_(term) == o_term).all()
        assert_same_state(env, s)
        if o_term.all():
            break
    env.close()


@pytest.mark.parametrize("name,game,rows,cols,n", MOVE, ids=[m[0] for m in MOVE])
def test_positions_round_trip_and_partial_playouts(L, name, game, rows, cols, n):
    n = min(n, 600)
    rng = np.random.default_rng(5)
    s = G.reset(game, rows, cols, n)
    G.rollout_from(s, seed=4, stop_ply=rng.integers(0, 120, n).astype(np.int16))
    env = L.Env(game, rows, cols, n, env_offset=2)
    push(env, s)
    assert_same_state(env, s)
    stop = (s.ply + rng.integers(1, 30, n)).astype(np.int16)
    s2 = s.copy()
    G.rollout_from(s2, seed=8, env_offset=2, stop_ply=stop)
    env.rollout(8, from_start=False, write_back=True, stop_ply=torch.from_numpy(stop).cuda())
    assert_same_state(env, s2)
    G.rollout_from(s2, seed=8, env_offset=2)
    env.rollout(8, from_start=False, write_back=True)
    assert_same_state(env, s2)
    env.close()


def test_illegal_actions(L):
    env = L.Env(G.DRAUGHTS, 8, 8, 3)
    # a man stepping backwards, a move from an empty cell, an action out of range
    acts = torch.tensor([42 * 64 + 51, 0 * 64 + 9, 64 * 64], dtype=torch.int32, device="cuda")
    rew, term = env.step(acts)
    torch.cuda.synchronize()
    assert (np_(term) == 1).all() and (np_(rew)[:, 0] == -1).all()
    assert env.counters()[0] == 3
    env.close()


def test_mixed_batch_with_move_games(L):
    n = 3000
    pool = [W.desc(8, 8, 8), W.desc(9, 8, 8), W.desc(10, 9, 9), W.desc(1, 6, 7), W.desc(0, 3, 3), W.desc(2, 8, 8)]
    d = np.array(pool, np.int32)[np.random.default_rng(2).integers(0, len(pool), n)]
    o, p = G.rollout_mixed(d, 6)
    out = torch.empty(n, dtype=torch.int8, device="cuda")
    plies = torch.empty(n, dtype=torch.int16, device="cuda")
    plan = L.ludax_mixed_plan_create(torch.from_numpy(d).cuda())
    L.ludax_mixed_plan_launch(plan, 6, out, plies)
    torch.cuda.synchronize()
    L.ludax_mixed_plan_destroy(plan)
    assert (np_(out) == o).all() and (np_(plies) == p).all()


@pytest.mark.parametrize("name,game,rows,cols,n,iters", [("wolf_sheep", G.WOLF_SHEEP, 8, 8, 64, 40),
                                                          ("draughts", G.DRAUGHTS, 8, 8, 48, 24),
                                                          ("hasami_shogi", G.HASAMI_SHOGI, 9, 9, 8, 8)])
def test_search_matches_oracle(L, name, game, rows, cols, n, iters):
    rng = np.random.default_rng(n)
    s = G.reset(game, rows, cols, n)
    G.rollout_from(s, seed=3, stop_ply=rng.integers(0, 40, n).astype(np.int16))
    env = L.Env(game, rows, cols, n, env_offset=4)
    push(env, s)
    act, vis, win = env.mcts_search(5, iters, stats=True)
    torch.cuda.synchronize()
    o_act, o_vis, o_win = G.mcts_search(s, 5, iters, env_offset=4)
    assert (np_(act) == o_act).all()
    assert (np_(vis).astype(np.uint32) == o_vis).all() and (np_(win).astype(np.uint32) == o_win).all()
    env.close()


@pytest.mark.parametrize("name,game,rows,cols,n,i1,i2", [("wolf_sheep", G.WOLF_SHEEP, 8, 8, 16, 30, 10),
                                                          ("draughts", G.DRAUGHTS, 8, 8, 6, 8, 8),
                                                          ("hasami_shogi", G.HASAMI_SHOGI, 9, 9, 2, 3, 3)])
def test_matches_match_oracle(L, name, game, rows, cols, n, i1, i2):
    env = L.Env(game, rows, cols, n, env_offset=1)
    got = [np_(t) for t in env.mcts_play(11, i1, i2)]
    want = G.mcts_play(game, rows, cols, n, 11, i1, i2, env_offset=1)
    for a, b in zip(got, want):
        assert (a == b).all()
    env.close()


def test_value_net_refuses_move_games(L):
    env = L.Env(G.DRAUGHTS, 8, 8, 4)
    x = torch.zeros(4, 256, dtype=torch.int16, device="cuda")
    with pytest.raises(L.LudaxError) as ei:
        L.ludax_pack_inputs(env.handle, x, 256)
    assert ei.value.status == -2
    env.close()
