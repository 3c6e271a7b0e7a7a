"""Pins of the oracle's line-game family (Gomoku 15x15, Pente 19x19,
Yavalath 61-cell hexagon; the paper's App. C) against closed forms,
hand-built positions and an independent numpy line scan."""
import numpy as np
import pytest

from oracle import games as G

PENTE_CENTRE = 9 * 19 + 9


def yav_cells():
    """(r, c) of the 61 cells in canonical order: rows 0..8, |r - c| <= 4."""
    return [(r, c) for r in range(9) for c in range(9) if abs(r - c) <= 4]


def test_yavalath_geometry():
    cells = yav_cells()
    assert len(cells) == 61 == G.num_cells(G.YAVALATH, 9, 9)
    lens = [sum(1 for r, c in cells if r == rr) for rr in range(9)]
    assert lens == [5, 6, 7, 8, 9, 8, 7, 6, 5]
    s = set(cells)
    nb = [sum((r + dr, c + dc) in s for dr, dc in ((0, 1), (0, -1), (1, 0), (-1, 0), (1, 1), (-1, -1)))
          for r, c in cells]
    assert nb.count(6) == 61 - 24 and min(nb) == 3   # 24 boundary cells, 6 corners with 3 neighbours
    assert nb.count(3) == 6


@pytest.mark.parametrize("game,rows,cols,depths", [
    (G.GOMOKU, 15, 15, [(1, 225), (2, 225 * 224)]),
    (G.PENTE, 19, 19, [(1, 1), (2, 360), (3, 360 * 359)]),
    (G.YAVALATH, 9, 9, [(1, 61), (2, 61 * 60), (3, 61 * 60 * 59)]),
])
def test_linegame_perft_closed_form(game, rows, cols, depths):
    # no line can be made and no capture is possible this early
    for d, want in depths:
        assert G.perft(game, rows, cols, d) == want


def play(game, rows, cols, moves):
    s = G.reset(game, rows, cols, 1)
    for m in moves:
        assert s.outcome[0] == -1, m
        G.step(s, [m])
    return s


def test_gomoku_exactly_five():
    C = 15
    # P1 builds a row 0..4 on row 7 while P2 plays far away: exactly five wins
    p2 = [0, 2, 4, 6, 8]
    moves = []
    for k in range(5):
        moves += [7 * C + k, p2[k]]
    s = play(G.GOMOKU, 15, 15, moves[:-1])
    assert s.outcome[0] == 1 and s.ply[0] == 9
    # six in a row does not win: P1 fills 7*C+0..4 except 2, plus 5, then closes the gap -> run of 6
    order = [7 * C + 0, 7 * C + 1, 7 * C + 3, 7 * C + 4, 7 * C + 5, 7 * C + 2]
    s = G.reset(G.GOMOKU, 15, 15, 1)
    for k, m in enumerate(order):
        G.step(s, [m])
        if k < len(order) - 1:
            G.step(s, [p2[k]])
    assert s.outcome[0] == -1 and (s.board[0, 7 * C:7 * C + 6] == 1).all()


def test_pente_centre_first_and_capture():
    s = G.reset(G.PENTE, 19, 19, 1)
    legal = G.legal(s)[0]
    assert legal.sum() == 1 and legal[PENTE_CENTRE]
    C = 19
    c0 = PENTE_CENTRE
    # P1 centre, P2 right of centre, P1 far, P2 two right, P1 three right: captures the pair
    s = play(G.PENTE, 19, 19, [c0, c0 + 1, 0, c0 + 2])
    G.step(s, [c0 + 3])
    assert s.board[0, c0 + 1] == 0 and s.board[0, c0 + 2] == 0
    assert s.passes[0] & 15 == 1          # one pair captured by P1
    # moving into a sandwich does not capture: P2 plays between two P1 stones
    s = play(G.PENTE, 19, 19, [c0, 40, c0 + 3, c0 + 1])
    G.step(s, [100])
    G.step(s, [c0 + 2])                   # P2 completes O O between X and X: no capture
    assert s.board[0, c0 + 1] == 2 and s.board[0, c0 + 2] == 2 and s.passes[0] == 0


def test_pente_ten_captures_win():
    # P1 to move with 4 pairs captured and a capture available -> 10 stones: win
    s = G.States(G.PENTE, 19, 19, 1)
    s.to_move[:] = 1
    s.ply[:] = 20
    s.outcome[:] = -1
    s.passes[:] = 4
    s.board[0, 5 * 19 + 5] = 1
    s.board[0, 5 * 19 + 6] = 2
    s.board[0, 5 * 19 + 7] = 2
    rew, term, _ = G.step(s, [5 * 19 + 8])
    assert term[0] and s.outcome[0] == 1 and s.passes[0] & 15 == 5


def test_yavalath_four_wins_three_loses():
    cells = yav_cells()
    idx = {rc: i for i, rc in enumerate(cells)}
    row4 = [idx[(4, c)] for c in range(9)]
    far = [idx[(0, 0)], idx[(8, 8)], idx[(0, 4)], idx[(8, 4)]]
    # P1: (4,0) (4,1) (4,3) then (4,2) completes four -> win
    s = play(G.YAVALATH, 9, 9, [row4[0], far[0], row4[1], far[1], row4[3], far[2]])
    G.step(s, [row4[2]])
    assert s.outcome[0] == 1
    # P1: (4,0) (4,1) then (4,2) makes three without four -> P1 loses
    s = play(G.YAVALATH, 9, 9, [row4[0], far[0], row4[1], far[1]])
    G.step(s, [row4[2]])
    assert s.outcome[0] == 2
    # three along the (1,1) axis also loses
    diag = [idx[(2, 2)], idx[(3, 3)], idx[(4, 4)]]
    s = play(G.YAVALATH, 9, 9, [diag[0], far[0], diag[1], far[1]])
    G.step(s, [diag[2]])
    assert s.outcome[0] == 2


def _runs(board2d, p, valid=None):
    """Maximal run lengths of player p along (0,1), (1,0), (1,1) and, when
    valid is None (square boards), (1,-1)."""
    H, Wd = board2d.shape
    dirs = [(0, 1), (1, 0), (1, 1)] + ([(1, -1)] if valid is None else [])
    inb = (lambda r, c: 0 <= r < H and 0 <= c < Wd and (valid is None or valid[r, c]))
    out = []
    for dr, dc in dirs:
        for r in range(H):
            for c in range(Wd):
                if not inb(r, c) or board2d[r, c] != p:
                    continue
                if inb(r - dr, c - dc) and board2d[r - dr, c - dc] == p:
                    continue
                k = 0
                while inb(r + k * dr, c + k * dc) and board2d[r + k * dr, c + k * dc] == p:
                    k += 1
                out.append(k)
    return out


def test_gomoku_random_games_consistent():
    out, plies, boards = G.rollout_start(G.GOMOKU, 15, 15, 40, seed=9, want_boards=True)
    for e in range(40):
        b = boards[e].reshape(15, 15)
        assert (b != 0).sum() == plies[e]
        if out[e] == 0:
            assert plies[e] == 225
        else:
            w = out[e]
            assert 5 in _runs(b, w) and 5 not in _runs(b, 3 - w)
            assert w == (1 if plies[e] % 2 == 1 else 2)


def test_yavalath_random_games_consistent():
    cells = yav_cells()
    valid = np.zeros((9, 9), bool)
    for r, c in cells:
        valid[r, c] = True
    out, plies, boards = G.rollout_start(G.YAVALATH, 9, 9, 300, seed=4, want_boards=True)
    for e in range(300):
        b2 = np.zeros((9, 9), np.int8)
        for i, (r, c) in enumerate(cells):
            b2[r, c] = boards[e, i]
        mover = 1 if plies[e] % 2 == 1 else 2
        rm = _runs(b2, mover, valid)
        if out[e] == mover:
            assert max(rm) >= 4
        elif out[e] == 3 - mover:
            assert max(rm) == 3
        else:
            assert out[e] == 0 and plies[e] == 61 and max(rm) <= 2


def test_pente_random_games_consistent():
    out, plies, boards = G.rollout_start(G.PENTE, 19, 19, 12, seed=3, want_boards=True)
    assert set(np.unique(out)) <= {1, 2}
    for e in range(12):
        b = boards[e].reshape(19, 19)
        w = out[e]
        assert w == (1 if plies[e] % 2 == 1 else 2)
        # the winner either has five in a row or has captured at least ten stones
        stones = {1: (b == 1).sum(), 2: (b == 2).sum()}
        placed_by_loser = plies[e] // 2
        captured_by_w = placed_by_loser - stones[3 - w]
        assert max(_runs(b, w)) >= 5 or captured_by_w >= 10


# ---------------------------------------------- parametric line game (m,n,k) --
LINE = 7


def line_game(L, exact=False, gravity=False, misere=False):
    return LINE | (L << 8) | ((1 if exact else 0) | (2 if gravity else 0) | (4 if misere else 0)) << 12


def test_line_game_closed_form_perft():
    # 4x4, line of 4: no game ends before ply 7, so perft = falling factorial
    want = 1
    for d in range(1, 6):
        want *= 16 - (d - 1)
        assert G.perft(line_game(4), 4, 4, d) == want
    # gravity on 5 columns of height 4: every column stays open for 4 plies
    for d in range(1, 5):
        assert G.perft(line_game(4, gravity=True), 4, 5, d) == 5 ** d


def test_misere_tic_tac_toe_loser_made_the_line():
    out, plies, boards = G.rollout_start(line_game(3, misere=True), 3, 3, 500, seed=8, want_boards=True)
    for e in range(500):
        b = boards[e].reshape(3, 3)
        mover = 1 if plies[e] % 2 == 1 else 2
        if out[e] == 0:
            assert plies[e] == 9 and max(_runs(b, 1)) < 3 and max(_runs(b, 2)) < 3
        else:
            assert out[e] == 3 - mover and max(_runs(b, mover)) >= 3


def test_exact_line_game_matches_gomoku_rule_on_small_board():
    # exactly-4 on 7x7: the winner has a maximal run of exactly 4 and the loser none
    out, plies, boards = G.rollout_start(line_game(4, exact=True), 7, 7, 300, seed=2, want_boards=True)
    for e in range(300):
        b = boards[e].reshape(7, 7)
        if out[e] in (1, 2):
            assert 4 in _runs(b, out[e]) and 4 not in _runs(b, 3 - out[e])
