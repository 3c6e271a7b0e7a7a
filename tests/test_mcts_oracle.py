"""Pins of the oracle's UCT agent and matches (App. F, GAVEL-like
evaluation: MCTS with UCB1 and a random rollout per iteration).  CPU only."""
import numpy as np
import pytest

from oracle import games as G

M64 = (1 << 64) - 1


def sm(x):
    """splitmix64 output for state x (Steele, Lea and Flood 2014)."""
    z = (x + 0x9E3779B97F4A7C15) & M64
    z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & M64
    z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & M64
    return z ^ (z >> 31)


def position(game, rows, cols, moves):
    s = G.reset(game, rows, cols, 1)
    for a in moves:
        _, _, err = G.step(s, np.array([a], np.int32))
        assert err[0] == 0
    return s


def batch_of(s, n):
    t = G.States(s.game, s.rows, s.cols, n)
    for k in ("board", "to_move", "ply", "passes", "outcome"):
        getattr(t, k)[:] = getattr(s, k)[0]
    return t


def test_visit_counts_add_up():
    s = G.reset(G.C4, 6, 7, 8)
    for iters in (1, 7, 50, 333):
        act, vis, win = G.mcts_search(s, 3, iters)
        assert (vis.sum(1) == iters).all()
        assert (win <= 2 * vis).all()
        # the chosen child has the most visits
        assert (vis[np.arange(8), act] == vis.max(1)).all()


def test_one_iteration_is_the_expansion_draw():
    """With one iteration the root gets one child: the k-th legal action,
    k = pick(sm(~key_0), n) with key_0 = sm(K ^ 0), K the search key."""
    s = G.reset(G.TTT, 3, 3, 64)
    act, _, _ = G.mcts_search(s, 11, 1, env_offset=100)
    for e in range(64):
        Km = sm(sm(11) ^ (100 + e))           # the match key
        K = sm(Km ^ (1 << 32))                # the search at ply 0
        k0 = sm(K ^ 0)
        k = ((sm(~k0 & M64) >> 32) * 9) >> 32
        assert act[e] == k


def test_full_expansion_visits_every_root_action_once():
    s = G.reset(G.TTT, 3, 3, 16)
    act, vis, win = G.mcts_search(s, 5, 9)
    assert (vis == 1).all()
    # every child played one rollout: its W is 0, 1 or 2; the move is the first best
    for e in range(16):
        best = np.flatnonzero(win[e] == win[e].max())[0]
        assert act[e] == best


@pytest.mark.parametrize("moves,win", [
    ([0, 3, 1, 4], 2),          # X: 0 1, O: 3 4 -> X completes the top row at 2
    ([4, 0, 8, 2, 6, 5], 7),    # X: 4 6 8, O: 0 2 5; X wins at 7 (row 6-7-8) instead of blocking 1
])
def test_ttt_takes_the_immediate_win(moves, win):
    s = batch_of(position(G.TTT, 3, 3, moves), 40)
    act, _, _ = G.mcts_search(s, 9, 200)
    assert (act == win).mean() >= 0.95


def test_ttt_blocks_the_immediate_loss():
    # X: 0 1, O: 4 -> O must block at 2
    s = batch_of(position(G.TTT, 3, 3, [0, 4, 1]), 40)
    act, _, _ = G.mcts_search(s, 2, 400)
    assert (act == 2).mean() >= 0.9


def test_connect_four_takes_the_win_and_blocks():
    # P1 stacks three in column 0 (cells 35, 28, 21), P2 plays column 6: P1 wins at 14
    s = batch_of(position(G.C4, 6, 7, [35, 41, 28, 34, 21, 27]), 30)
    act, _, _ = G.mcts_search(s, 4, 300)
    assert (act == 14).mean() >= 0.95
    # P2 to move with P1 threatening 14: P2 blocks
    s = batch_of(position(G.C4, 6, 7, [35, 41, 28, 34, 21]), 30)
    act, _, _ = G.mcts_search(s, 6, 400)
    assert (act == 14).mean() >= 0.9


def test_stronger_agent_beats_a_one_iteration_agent():
    out, plies, agency, cov = G.mcts_play(G.C4, 6, 7, 24, 1, 200, 1)
    assert (out == 1).mean() >= 0.9
    out, plies, agency, cov = G.mcts_play(G.C4, 6, 7, 24, 2, 1, 200)
    assert (out == 2).mean() >= 0.9
    out, *_ = G.mcts_play(G.TTT, 3, 3, 40, 3, 400, 1)
    assert (out == 2).sum() == 0


@pytest.mark.parametrize("game,rows,cols,start", [(G.TTT, 3, 3, 0), (G.C4, 6, 7, 0), (G.HEX, 5, 5, 0),
                                                  (G.OTHELLO, 8, 8, 4), (7 | (4 << 8) | (2 << 12), 5, 6, 0)])
def test_match_invariants(game, rows, cols, start):
    out, plies, agency, cov = G.mcts_play(game, rows, cols, 12, 7, 30, 20)
    assert ((out >= 0) & (out <= 2)).all()
    assert (agency <= plies).all() and (agency >= 1).all()
    if game == G.OTHELLO:
        assert (cov <= 64).all() and (cov >= 4).all()
    else:
        # stones are never removed: every ply occupies a new cell
        assert (cov == plies).all()
    if game == G.C4:
        assert (agency >= plies - 6).all()   # a single legal column happens only near the end


def test_pente_coverage_counts_captured_cells():
    out, plies, agency, cov = G.mcts_play(G.PENTE, 19, 19, 2, 3, 4, 4)
    assert (cov <= plies).all() and (cov >= 1).all()
    assert ((out >= 0) & (out <= 2)).all()
