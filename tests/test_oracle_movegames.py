"""Pins of the oracle's move games (App. C): Wolf and Sheep, English
Draughts, Dai Hasami Shogi.  Action = from * cells + to.  CPU only."""
import numpy as np
import pytest

from oracle import games as G


def state(game, rows, cols, cells, to_move=1, ply=10, pending=-1):
    s = G.States(game, rows, cols, 1)
    for i, v in cells.items():
        s.board[0, i] = v
    s.to_move[0] = to_move
    s.ply[0] = ply
    s.passes[0] = pending + 1 if game == G.DRAUGHTS else 0
    s.outcome[0] = -1
    return s


def legal_moves(s):
    N = s.board.shape[1]
    return [(a // N, a % N) for a in np.flatnonzero(G.legal(s)[0])]


def play(s, frm, to):
    N = s.board.shape[1]
    _, _, err = G.step(s, np.array([frm * N + to], np.int32))
    assert err[0] == 0


# ----------------------------------------------------------- Draughts --
def test_draughts_perft_matches_the_published_counts():
    # English draughts perft from the start (a multi-capture is one move)
    want = [7, 49, 302, 1469, 7361, 36768, 179740, 845931]
    assert [G.perft_turns(G.DRAUGHTS, 8, 8, d) for d in range(1, 9)] == want
    # per ply, a multi-capture is several actions: equal until the first one
    assert [G.perft(G.DRAUGHTS, 8, 8, d) for d in range(1, 7)] == want[:6]


def test_draughts_capture_is_forced_and_continues():
    # P1 man on 45 (5,5), P2 men on 36 (4,4) and 20 (2,4); P1 also has a free man on 47
    s = state(G.DRAUGHTS, 8, 8, {45: 1, 47: 1, 36: 2, 20: 2, 0: 2})
    assert legal_moves(s) == [(45, 27)]           # the hop is the only legal action
    play(s, 45, 27)
    assert s.board[0, 36] == 0 and s.to_move[0] == 1 and s.passes[0] == 27 + 1   # extra turn, piece 27
    assert legal_moves(s) == [(27, 13)]
    play(s, 27, 13)
    assert s.board[0, 20] == 0 and s.to_move[0] == 2 and s.passes[0] == 0


def test_draughts_promotion_and_king_moves():
    s = state(G.DRAUGHTS, 8, 8, {10: 1, 63: 2})
    play(s, 10, 1)                                 # (1,2) -> (0,1): the man is crowned
    assert s.board[0, 1] == 3
    s = state(G.DRAUGHTS, 8, 8, {27: 3, 63: 2})    # a P1 king in the centre moves in all 4 directions
    assert sorted(t for f, t in legal_moves(s)) == [18, 20, 34, 36]


def test_draughts_side_without_moves_loses():
    # P2's only man is captured: P1 wins
    s = state(G.DRAUGHTS, 8, 8, {45: 1, 36: 2})
    play(s, 45, 27)
    assert s.outcome[0] == 1
    # P2 man on 56 (7,0) cannot move (men only go down for P2): after P1 moves, P1 wins
    s = state(G.DRAUGHTS, 8, 8, {56: 2, 43: 1})
    play(s, 43, 34)
    assert s.outcome[0] == 1


# ----------------------------------------------------- Wolf and Sheep --
def ws_moves(sheep, wolf, p):
    out = []
    if p == 1:
        for s in sorted(sheep):
            r, c = divmod(s, 8)
            for dc in (-1, 1):
                t = (r - 1) * 8 + c + dc
                if r - 1 >= 0 and 0 <= c + dc < 8 and t not in sheep and t != wolf:
                    out.append((s, t))
    else:
        r, c = divmod(wolf, 8)
        for dr in (-1, 1):
            for dc in (-1, 1):
                t = (r + dr) * 8 + c + dc
                if 0 <= r + dr < 8 and 0 <= c + dc < 8 and t not in sheep:
                    out.append((wolf, t))
    return sorted(out)


def ws_perft(sheep, wolf, p, depth):
    """Independent brute force: the rules written out on cell sets."""
    if depth == 0:
        return 1
    total = 0
    for f, t in ws_moves(sheep, wolf, p):
        sh, wo = (sheep - {f}) | {t} if p == 1 else sheep, t if p == 2 else wolf
        over = (p == 2 and t // 8 == 7) or not ws_moves(sh, wo, 3 - p)
        if over:
            total += 1 if depth == 1 else 0    # a finished game has no deeper leaves
        else:
            total += ws_perft(sh, wo, 3 - p, depth - 1)
    return total


def test_wolf_and_sheep_perft_against_brute_force():
    sheep, wolf = {56, 58, 60, 62}, 3
    for d in range(1, 7):
        assert G.perft(G.WOLF_SHEEP, 8, 8, d) == ws_perft(sheep, wolf, 1, d)


def test_wolf_and_sheep_end_rules():
    s = state(G.WOLF_SHEEP, 8, 8, {49: 2, 56: 1})   # the wolf on (6,1), a sheep on (7,0)
    s.to_move[0] = 2
    play(s, 49, 58)
    assert s.outcome[0] == 2                                  # reached the bottom row
    # the wolf in the corner 7 (0,7) with only (1,6) free: a sheep closes it
    s = state(G.WOLF_SHEEP, 8, 8, {7: 2, 21: 1})
    play(s, 21, 14)
    assert s.outcome[0] == 1


# --------------------------------------------------- Dai Hasami Shogi --
def test_hasami_first_moves_counted_by_hand():
    # 9 pieces of row 7 slide up 1..5 cells, 9 pieces of row 8 hop over row 7
    assert G.perft(G.HASAMI_SHOGI, 9, 9, 1) == 9 * 5 + 9
    s = G.reset(G.HASAMI_SHOGI, 9, 9, 1)
    mv = legal_moves(s)
    assert (72, 54) in mv and (63, 18) in mv and (63, 9) not in mv


def test_hasami_custodial_captures():
    # P2 pieces on 40 (4,4) and 41 (4,5), P1 on 42 (4,6); P1 slides 37 -> 39 (4,3): both removed
    s = state(G.HASAMI_SHOGI, 9, 9, {40: 2, 41: 2, 42: 1, 37: 1, 0: 2, 80: 1})
    play(s, 37, 39)
    assert s.board[0, 40] == 0 and s.board[0, 41] == 0
    # moving between two opposing pieces is safe
    s = state(G.HASAMI_SHOGI, 9, 9, {39: 2, 41: 2, 31: 1, 0: 2, 80: 1})
    play(s, 31, 40)
    assert s.board[0, 40] == 1 and s.board[0, 39] == 2 and s.board[0, 41] == 2


def test_hasami_corner_capture():
    # P2 in corner 0, P1 on 9 (1,0); P1 moves 19 -> 1 (0,1): the corner piece is removed
    s = state(G.HASAMI_SHOGI, 9, 9, {0: 2, 9: 1, 19: 1, 40: 2, 80: 1})
    play(s, 19, 1)
    assert s.board[0, 0] == 0


def test_hasami_five_in_a_row_outside_the_home_rows():
    # P1 has 4 in row 4 and slides a fifth in: win
    s = state(G.HASAMI_SHOGI, 9, 9, {36: 1, 37: 1, 38: 1, 39: 1, 49: 1, 0: 2, 10: 2})
    play(s, 49, 40)
    assert s.outcome[0] == 1
    # the same five on P1's starting row 7 do not count
    s = state(G.HASAMI_SHOGI, 9, 9, {63: 1, 64: 1, 65: 1, 66: 1, 76: 1, 0: 2, 10: 2})
    play(s, 76, 67)
    assert s.outcome[0] == -1


@pytest.mark.parametrize("game,rows,cols", [(G.WOLF_SHEEP, 8, 8), (G.DRAUGHTS, 8, 8), (G.HASAMI_SHOGI, 9, 9)])
def test_move_game_playouts_are_consistent(game, rows, cols):
    out, plies, boards = G.rollout_start(game, rows, cols, 200, 3, want_boards=True)
    assert ((out >= 0) & (out <= 3)).all() and (plies <= 200).all()
    assert (plies[out == 3] == 200).all()          # a capped game used all 200 turns (a win on the 200th counts)
    if game == G.WOLF_SHEEP:
        assert (out != 0).all()                   # no draws
