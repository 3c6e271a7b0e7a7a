"""UCT agents and matches on the GPU (App. F) against the oracle, element
by element: chosen actions, the root children's visit counts and half-point
rewards, and whole matches (outcome, plies, agency, coverage)."""
import math

import numpy as np
import pytest
import torch

from oracle import games as G
from paper_2506_22609_b300 import gavel

pytestmark = pytest.mark.gpu

LINE_4X5_GRAVITY = 7 | (4 << 8) | (2 << 12)
LINE_4X4_MISERE = 7 | (3 << 8) | (4 << 12)

# (name, game, rows, cols, envs, iterations)
SEARCH_CASES = [
    ("ttt", G.TTT, 3, 3, 300, 64), ("c4", G.C4, 6, 7, 200, 64), ("othello", G.OTHELLO, 8, 8, 96, 32),
    ("hex5", G.HEX, 5, 5, 96, 48), ("hex11", G.HEX, 11, 11, 24, 40), ("gomoku", G.GOMOKU, 15, 15, 12, 24),
    ("pente", G.PENTE, 19, 19, 8, 16), ("yavalath", G.YAVALATH, 9, 9, 24, 32),
    ("line_gravity", LINE_4X5_GRAVITY, 4, 5, 96, 48), ("line_misere", LINE_4X4_MISERE, 4, 4, 96, 48),
]


def env_for(L, game, rows, cols, n, **kw):
    if game & 0xFF == 7:
        return L.Env("line", rows, cols, n, line=(game >> 8) & 15, flags=(game >> 12) & 7, **kw)
    return L.Env(game, rows, cols, n, **kw)


def push(env, s):
    env.set_state(*(torch.from_numpy(x) for x in (s.board, s.to_move, s.ply, s.passes, s.outcome)))


@pytest.mark.parametrize("name,game,rows,cols,n,iters", SEARCH_CASES, ids=[c[0] for c in SEARCH_CASES])
def test_search_matches_oracle(L, name, game, rows, cols, n, iters):
    rng = np.random.default_rng(n + rows)
    s = G.reset(game, rows, cols, n)
    # positions along random games (some envs stay at the start, some end)
    G.rollout_from(s, seed=5, stop_ply=rng.integers(0, rows * cols // 2 + 2, n).astype(np.int16))
    env = env_for(L, game, rows, cols, n, env_offset=7)
    push(env, s)
    c = math.sqrt(2.0)
    act, vis, win = env.mcts_search(13, iters, c, stats=True)
    torch.cuda.synchronize()
    o_act, o_vis, o_win = G.mcts_search(s, 13, iters, c, env_offset=7)
    assert (act.cpu().numpy() == o_act).all()
    assert (vis.cpu().numpy().astype(np.uint32) == o_vis).all()
    assert (win.cpu().numpy().astype(np.uint32) == o_win).all()
    live = s.outcome == -1
    assert (o_vis[live].sum(1) == iters).all() and (o_act[~live] == -1).all()
    env.close()


@pytest.mark.parametrize("c", [0.0, 0.5, 3.0])
def test_search_exploration_constant(L, c):
    n = 64
    s = G.reset(G.C4, 6, 7, n)
    G.rollout_from(s, seed=2, stop_ply=np.full(n, 6, np.int16))
    env = env_for(L, G.C4, 6, 7, n)
    push(env, s)
    act, vis, win = env.mcts_search(4, 80, c, stats=True)
    torch.cuda.synchronize()
    o_act, o_vis, o_win = G.mcts_search(s, 4, 80, c)
    assert (act.cpu().numpy() == o_act).all() and (vis.cpu().numpy().astype(np.uint32) == o_vis).all()
    env.close()


# (name, game, rows, cols, matches, iters P1, iters P2)
PLAY_CASES = [
    ("ttt", G.TTT, 3, 3, 96, 100, 100), ("c4", G.C4, 6, 7, 24, 40, 20), ("othello", G.OTHELLO, 8, 8, 8, 12, 6),
    ("hex5", G.HEX, 5, 5, 16, 30, 30), ("line_misere", LINE_4X4_MISERE, 4, 4, 24, 24, 12),
    ("line_gravity", LINE_4X5_GRAVITY, 4, 5, 24, 20, 20), ("yavalath", G.YAVALATH, 9, 9, 4, 8, 8),
    ("gomoku", G.GOMOKU, 15, 15, 2, 4, 4), ("pente", G.PENTE, 19, 19, 2, 3, 3),
]


@pytest.mark.parametrize("name,game,rows,cols,n,i1,i2", PLAY_CASES, ids=[c[0] for c in PLAY_CASES])
def test_matches_match_oracle(L, name, game, rows, cols, n, i1, i2):
    env = env_for(L, game, rows, cols, n, env_offset=3)
    out, plies, agency, cov = (t.cpu().numpy() for t in env.mcts_play(21, i1, i2))
    o = G.mcts_play(game, rows, cols, n, 21, i1, i2, env_offset=3)
    for got, want in zip((out, plies, agency, cov), o):
        assert (got == want).all()
    env.close()


def test_match_write_back_and_from_current_state(L):
    n = 16
    env = env_for(L, G.C4, 6, 7, n)
    out, plies, _, _ = env.mcts_play(8, 10, 10, write_back=True)
    b, tm, ply, ps, oc = env.get_state()
    torch.cuda.synchronize()
    assert (ply.cpu().numpy() == plies.cpu().numpy()).all() and (oc.cpu().numpy() == out.cpu().numpy()).all()
    # a finished match played again from its stored state stays as it is
    out2, plies2, agency2, _ = env.mcts_play(8, 10, 10, from_start=False)
    assert (out2.cpu() == out.cpu()).all() and (plies2.cpu() == plies.cpu()).all() and (agency2.cpu() == 0).all()
    env.close()


def test_argument_validation(L):
    env = env_for(L, G.TTT, 3, 3, 4)
    for iters, c in ((0, 1.0), (L.LUDAX_MCTS_MAX_ITERS + 1, 1.0), (10, -1.0), (10, float("nan"))):
        with pytest.raises(L.LudaxError) as ei:
            env.mcts_search(1, iters, c)
        assert ei.value.status == -1
    with pytest.raises(L.LudaxError):
        env.mcts_play(1, 5, 0)
    env.close()


def test_gavel_evaluation_runs_on_the_gpu(L):
    from paper_2506_22609_b300 import dsl

    res = gavel.evaluate(dsl.library()["tic_tac_toe"], matches=32, iters=60, weak_iters=10, seed=1)
    assert res["playable"] and 0.0 <= res["gavel_score"] <= 1.0
    for k in gavel.HEURISTICS:
        assert -1.0 <= res[k] <= 1.0
    # TTT between equal agents: complete, every cell coverable, agency high
    assert res["completion"] == 1.0 and res["agency"] > 0.8


def test_mixed_matches_match_oracle(L):
    from paper_2506_22609_b300 import workloads as W

    groups = [(G.TTT, 3, 3, 12), (G.C4, 6, 7, 6), (G.HEX, 5, 5, 4), (LINE_4X4_MISERE, 4, 4, 6),
              (G.OTHELLO, 8, 8, 3), (G.YAVALATH, 9, 9, 2), (G.GOMOKU, 15, 15, 1), (G.PENTE, 19, 19, 1),
              (LINE_4X5_GRAVITY, 4, 5, 4)]

    def desc_of(game, rows, cols):
        if game & 0xFF == 7:
            return L.LUDAX_DESC_LINE(rows, cols, (game >> 8) & 15, (game >> 12) & 7)
        return W.desc(game, rows, cols)

    desc, iters, who = [], [], []
    rng = np.random.default_rng(4)
    for game, rows, cols, k in groups:
        for _ in range(k):
            desc.append(desc_of(game, rows, cols))
            iters.append((int(rng.integers(2, 30)), int(rng.integers(2, 30))))
            who.append((game, rows, cols))
    # shuffle so that neighbouring warps play different games
    order = rng.permutation(len(desc))
    desc = [desc[i] for i in order]
    iters = [iters[i] for i in order]
    who = [who[i] for i in order]
    n, off, seed = len(desc), 40, 12
    out = torch.empty(n, dtype=torch.int8, device="cuda")
    plies, agency, cov = (torch.empty(n, dtype=torch.int16, device="cuda") for _ in range(3))
    L.ludax_mcts_play_mixed(np.array(desc, np.int32), np.array(iters, np.int32), off, seed, 2 ** 0.5, out, plies,
                            agency, cov)
    torch.cuda.synchronize()
    got = [t.cpu().numpy() for t in (out, plies, agency, cov)]
    for e in range(n):
        game, rows, cols = who[e]
        want = G.mcts_play(game, rows, cols, 1, seed, iters[e][0], iters[e][1], env_offset=off + e)
        for g_arr, w_arr in zip(got, want):
            assert g_arr[e] == w_arr[0], (e, who[e])
    # invalid descriptors and iteration counts are caught on the host
    bad = np.array(desc, np.int32)
    bad[3] = W.desc(3, 12, 12)
    with pytest.raises(L.LudaxError) as ei:
        L.ludax_mcts_play_mixed(bad, np.array(iters, np.int32), 0, 1, 1.0, out)
    assert ei.value.status == -3 and ei.value.bad_index == 3
    it = np.array(iters, np.int32)
    it[5, 1] = 0
    with pytest.raises(L.LudaxError) as ei:
        L.ludax_mcts_play_mixed(np.array(desc, np.int32), it, 0, 1, 1.0, out)
    assert ei.value.status == -1 and ei.value.bad_index == 5


def test_gavel_single_and_many_agree(L):
    from paper_2506_22609_b300 import dsl

    lib = dsl.library()
    one = gavel.evaluate(lib["connect_four"], matches=8, iters=20, weak_iters=5, seed=3)
    many = gavel.evaluate_many({"a": lib["tic_tac_toe"], "c4": lib["connect_four"]}, 8, 20, 5, 3)
    # the same game at different global match indices gives different matches; at the
    # same indices, the same ones
    first = many["c4"]["first_match"]
    desc = [dsl.descriptor(lib["connect_four"])] * 8
    out = torch.empty(8, dtype=torch.int8, device="cuda")
    L.ludax_mcts_play_mixed(np.array(desc, np.int32), np.array([(20, 20)] * 8, np.int32), first, 3, 2 ** 0.5, out)
    o = G.mcts_play(G.C4, 6, 7, 8, 3, 20, 20, env_offset=first)[0]
    assert (out.cpu().numpy() == o).all()
    assert 0.0 <= one["gavel_score"] <= 1.0
