"""Game-description compiler: reader, grammar-directed elaboration, lowering
to descriptors (Sec. 3, Sec. 4, App. B).  CPU only."""
import numpy as np
import pytest

from oracle import games as G
from paper_2506_22609_b300 import dsl
from paper_2506_22609_b300 import workloads as W
from paper_2506_22609_b300.ludax import LUDAX_DESC_LINE

LIB = dsl.library()


def oracle_gid(spec):
    """The oracle's game id for a compiled spec (line games carry L and flags)."""
    return spec.game if spec.game != dsl.GAME_LINE else 7 | (spec.line << 8) | (spec.flags << 12)


# ------------------------------------------------------------------ reader --
def test_reader_tokens_comments_keywords():
    S, K = dsl.Sym, dsl.Kw
    f = dsl.read('(a "b c" 12 // comment (\n  k: v k2:(x y) k3:true)')
    assert f == [S("a"), dsl.Str("b c"), 12, K("k"), S("v"), K("k2"), [S("x"), S("y")], K("k3"), S("true")]


@pytest.mark.parametrize("text,where", [("(a (b)", "line 1"), ("(a))", "line 1"), ("(a)\n(b)", ""),
                                        ('(a "open)', "line 1"), ("(a\n\n(b", "line 3")])
def test_reader_errors_name_the_line(text, where):
    with pytest.raises(dsl.DslError) as ei:
        dsl.read(text)
    assert ei.value.path == where


# ----------------------------------------------------------- the library --
EXPECTED = {
    "tic_tac_toe": W.desc(0, 3, 3),
    "connect_four": W.desc(1, 6, 7),
    "reversi": W.desc(2, 8, 8),
    "hex": W.desc(3, 11, 11),
    "gomoku": W.desc(4, 15, 15),
    "pente": W.desc(5, 19, 19),
    "yavalath": W.desc(6, 9, 9),
    "misere_tic_tac_toe": LUDAX_DESC_LINE(3, 3, 3, dsl.LINE_MISERE),
    "connect_five_9x12": LUDAX_DESC_LINE(9, 12, 5, dsl.LINE_EXACT | dsl.LINE_GRAVITY),
    "tic_tac_four_5x5": LUDAX_DESC_LINE(5, 5, 4, 0),
    "wolf_and_sheep": W.desc(8, 8, 8),
    "english_draughts": W.desc(9, 8, 8),
    "dai_hasami_shogi": W.desc(10, 9, 9),
}


def test_library_compiles_to_the_expected_descriptors():
    assert set(LIB) == set(EXPECTED)
    for name, text in LIB.items():
        assert dsl.descriptor(text) == EXPECTED[name], name


def test_generic_lowering_of_dedicated_kernels():
    assert dsl.descriptor(LIB["tic_tac_toe"], specialize=False) == LUDAX_DESC_LINE(3, 3, 3, 0)
    assert dsl.descriptor(LIB["connect_four"], specialize=False) == LUDAX_DESC_LINE(6, 7, 4, dsl.LINE_GRAVITY)
    # 15 x 16 padded cells do not fit the parametric kernel: Gomoku keeps its own
    assert dsl.descriptor(LIB["gomoku"], specialize=False) == W.desc(4, 15, 15)


@pytest.mark.parametrize("name,seed", [("tic_tac_toe", 4), ("connect_four", 9)])
def test_specialised_and_generic_descriptors_play_identically(name, seed):
    """Two independent oracle rule sets (the dedicated game and the parametric
    line game) must give the same playouts for the same compiled text: pins
    the compiler's mapping of destination and end rules onto flags."""
    a = dsl.compile_game(LIB[name])
    b = dsl.compile_game(LIB[name], specialize=False)
    assert a.game != b.game
    n = 3000
    oa, pa, ba = G.rollout_start(oracle_gid(a), a.rows, a.cols, n, seed, want_boards=True)
    ob, pb, bb = G.rollout_start(oracle_gid(b), b.rows, b.cols, n, seed, want_boards=True)
    assert (oa == ob).all() and (pa == pb).all() and (ba == bb).all()
    oc, pc = G.rollout_mixed(np.array([a.desc, b.desc] * (n // 2), np.int32), seed)
    assert (oc[0::2] == oa[0::2]).all() and (oc[1::2] == oa[1::2]).all()


def test_library_runs_through_the_oracle_mixed_batch():
    d = np.array([EXPECTED[k] for k in sorted(EXPECTED)] * 50, np.int32)
    o, p = G.rollout_mixed(d, 17)
    move = np.isin(d & 0xFF, (8, 9, 10))
    assert ((o >= 0) & (o <= 2)).all() or ((o == 3) <= move).all()   # only move games stop at their 200-ply cap
    assert ((o >= 0) & (o <= 3)).all() and (p > 0).all() and (p[o == 3] == 200).all()


# ----------------------------------------------------------- normalisation --
TEMPLATE = """
(game "t" (players 2)
  (equipment (board {board}) (pieces ("s" both)))
  (rules (play (repeat (P1 P2) (place "s" (destination {dest}))))
    (end {end})))
"""


def mk(board="(square 3)", dest="(empty)", end='(if (line "s" 3) (mover win)) (if (full_board) (draw))'):
    return TEMPLATE.format(board=board, dest=dest, end=end)


@pytest.mark.parametrize("end", [
    '(if (line "s" 3) (mover win)) (if (full_board) (draw))',
    '(if (>= (line "s" 3) 1) (opponent lose)) (if (full_board) (draw))',
    '(if (line "s" 3 orientation: any player: mover) (mover win)) (if (full_board) (draw))',
    '(if (and (line "s" 3) (line "s" 3)) (mover win)) (if (full_board) (draw))',
])
def test_equivalent_end_rules_give_the_same_descriptor(end):
    assert dsl.descriptor(mk(end=end)) == W.desc(0, 3, 3)


@pytest.mark.parametrize("dest", [
    "(and (empty) (or (edge bottom) (adjacent (occupied) direction: up)))",
    "(and (or (adjacent (occupied) direction:up) (edge bottom)) (empty))",
    "(and (empty) (or (edge bottom) (or (adjacent (occupied) direction: (up)))))",
])
def test_gravity_destination_forms(dest):
    s = dsl.compile_game(mk(board="(rectangle 5 6)", dest=dest,
                            end='(if (line "s" 4) (mover win)) (if (full_board) (draw))'))
    assert (s.game, s.rows, s.cols, s.line, s.flags) == (dsl.GAME_LINE, 5, 6, 4, dsl.LINE_GRAVITY)


HEX_P1 = '(and (mover_is P1) (connected "stone" ((edge top) (edge bottom))))'
HEX_P2 = '(and (mover_is P2) (connected "stone" ((edge left) (edge right))))'


def hex_text(end, n=11):
    return (f'(game "h" (players 2) (equipment (board (hex_rectangle {n} {n})) (pieces ("stone" both)))'
            f' (rules (play (repeat (P1 P2) (place "stone" (destination (empty))))) (end {end})))')


def test_hex_end_rule_forms_and_sizes():
    forms = [
        f"(if {HEX_P1} (mover win)) (if {HEX_P2} (mover win))",
        f"(if {HEX_P2} (mover win)) (if {HEX_P1} (mover win))",
        f"(if (or {HEX_P2} {HEX_P1}) (mover win))",
        # operands of and / or in either order, edges listed in either order
        '(if (and (connected "stone" ((edge bottom) (edge top))) (mover_is P1)) (mover win))'
        '(if (and (connected "stone" ((edge right) (edge left))) (mover_is P2)) (mover win))',
    ]
    for end in forms:
        assert dsl.descriptor(hex_text(end)) == W.desc(3, 11, 11), end
    for n in (2, 7, 9):
        assert dsl.descriptor(hex_text(forms[0], n)) == W.desc(3, n, n)


def test_yavalath_three_rule_exact_or_not():
    t = LIB["yavalath"].replace('(line "stone" 3)', '(line "stone" 3 exact: true)')
    assert dsl.descriptor(t) == W.desc(6, 9, 9)


@pytest.mark.parametrize("rows,cols,L,exact,misere", [(3, 3, 3, 1, 0), (4, 7, 4, 0, 1), (10, 10, 5, 1, 1),
                                                      (1, 8, 3, 0, 0), (7, 15, 6, 0, 0)])
def test_mnk_family(rows, cols, L, exact, misere):
    board = f"(square {rows})" if rows == cols else f"(rectangle {rows} {cols})"
    ex = " exact: true" if exact else ""
    res = "(mover lose)" if misere else "(mover win)"
    s = dsl.compile_game(mk(board=board, end=f'(if (line "s" {L}{ex}) {res}) (if (full_board) (draw))'))
    flags = (dsl.LINE_EXACT if exact else 0) | (dsl.LINE_MISERE if misere else 0)
    if (rows, cols, L, flags) == (3, 3, 3, 0):
        assert s.game == dsl.GAME_TTT
    else:
        assert s.desc == LUDAX_DESC_LINE(rows, cols, L, flags)


# ------------------------------------------------------------- rejections --
@pytest.mark.parametrize("text,path,words", [
    (mk(dest='(empty)').replace('(place "s" (destination (empty)))', '(move (step "s" direction: up))'),
     "equipment/board", "move-game kernels"),
    (mk(end='(if (pattern "s" (square 2)) (mover win)) (if (full_board) (draw))'),
     "game/rules/end/if[0]", "no kernel family implements"),
    (mk(end='(if (line "t" 3) (mover win)) (if (full_board) (draw))'), "game/rules/end/if[0]", "not declared"),
    (mk(end='(if (line "s" 3 orientation: orthogonal) (mover win)) (if (full_board) (draw))'), "rules/end/if[0]",
     "every orientation"),
    (mk(end='(if (line "s" 3) (mover win))'), "rules/end", "full_board"),
    (mk(board="(square 12)", end='(if (line "s" 5) (mover win)) (if (full_board) (draw))'), "equipment/board",
     "larger than"),
    (mk(board="(hexagon 7)"), "equipment/board", "(hexagon 9)"),
    (mk(board="(hexagon 8)"), "game/equipment/board", "odd"),
    (mk(dest="(column 2)"), "rules/play/place/destination", "supported destinations"),
    (mk(dest="(frobnicate)"), "game/rules/play/phase[0]/place/destination", "unknown mask"),
    (mk().replace("(players 2)", "(players 3)"), "players", "two-player"),
    (mk().replace("(repeat (P1 P2)", "(repeat (P2 P1)"), "rules/play", "P1 first"),
    (mk(end='(if (line "s" 3 exclude: (edge top)) (mover win)) (if (full_board) (draw))'), "rules/end/if[0]",
     "every orientation"),
    (mk(end='(if (line "s" 3) (mover win) extra) (if (full_board) (draw))'), "game/rules/end/if[0]", "expected (if"),
    (LIB["reversi"].replace("(28 35)", "(27 35)"), "rules/start", "28 and 35"),
    (LIB["reversi"].replace("(force_pass)", ""), "rules/play", "force_pass"),
    (LIB["pente"].replace("(>= (score mover) 10)", "(>= (score mover) 8)"), "rules/end", "score of 10"),
    (LIB["pente"].replace('(custodial "stone" 2)', '(custodial "stone" 3)'), "rules/play/phase[1]", "custodial"),
    (LIB["yavalath"].replace('(if (line "stone" 3) (mover lose))', ""), "rules/end", "line of 3 loses"),
    (LIB["hex"].replace("(edge bottom)", "(edge right)"), "rules/end", "connects"),
    (LIB["hex"].replace("11 11", "12 12"), "equipment/board", "2 <= n <= 11"),
])
def test_rejections_name_the_node(text, path, words):
    with pytest.raises(dsl.DslError) as ei:
        dsl.compile_game(text)
    assert ei.value.path == path and words in str(ei.value), str(ei.value)


# ------------------------------------------------------------ move games --
def test_move_game_equivalent_forms():
    ws = LIB["wolf_and_sheep"]
    # the sheep's forward diagonals written absolutely; the end rules in the other order
    alt = ws.replace("(step \"sheep\" direction: (forward_left forward_right))",
                     "(step \"sheep\" direction: (up_right up_left))")
    alt = alt.replace("""            (if (and (mover_is P2) (last_move_in (edge bottom))) (mover win))
            (if (no_legal_actions) (mover win))""", """            (if (no_legal_actions) (mover win))
            (if (and (last_move_in (edge bottom)) (mover_is P2)) (mover win))""")
    assert alt != ws and dsl.descriptor(alt) == W.desc(8, 8, 8)
    # one hop over any piece is the same as hops over the mover's and the opponent's
    hs = LIB["dai_hasami_shogi"].replace("""                        (hop "piece" direction: orthogonal hop_over: mover)
                        (hop "piece" direction: orthogonal hop_over: opponent))""",
                                         """                        (hop "piece" direction: orthogonal))""")
    assert hs != LIB["dai_hasami_shogi"] and dsl.descriptor(hs) == W.desc(10, 9, 9)
    # no set_forward: P1 moves up by default
    dr = LIB["english_draughts"].replace("(players 2 (set_forward (P1 up) (P2 down)))", "(players 2)")
    assert dsl.descriptor(dr) == W.desc(9, 8, 8)


@pytest.mark.parametrize("name,old,new,path,words", [
    ("english_draughts", '(promote "pawn" "king" (edge forward))', '(promote "pawn" "king" (edge backward))',
     "rules/play/effects", "promote"),
    ("english_draughts", "priority: 1", "priority: 0", "rules/play", "priority"),
    ("english_draughts", "(set_forward (P1 up) (P2 down))", "(set_forward (P1 down) (P2 up))", "players",
     "set_forward"),
    ("wolf_and_sheep", '(place "wolf" P2 (3))', '(place "wolf" P2 (5))', "rules/start", "wolf on 3"),
    ("dai_hasami_shogi", "hop_over: mover)", "hop_over: mover capture: true)", "rules/play", "no capture"),
    ("dai_hasami_shogi", "((row 7) (row 8))", "((row 6) (row 7))", "rules/end", "home rows"),
    ("dai_hasami_shogi", '(capture (corner_custodial "piece"))', '(capture (custodial "piece" 1))',
     "rules/play/effects", "corners"),
])
def test_move_game_rejections(name, old, new, path, words):
    text = LIB[name]
    assert old in text
    with pytest.raises(dsl.DslError) as ei:
        dsl.compile_game(text.replace(old, new, 1))
    assert ei.value.path == path and words in str(ei.value), str(ei.value)


def test_move_mechanics_parse_into_the_normal_form():
    g = dsl.elaborate(dsl.read(LIB["english_draughts"]))
    kind, order, mech, force_pass = g["play"][0]
    assert mech[0] == "move" and len(mech[1]) == 4 and not force_pass
    assert ("hop", "pawn", ("forward_left", "forward_right"), None, "opponent", True, 0) in mech[1]
    assert mech[2][0] == ("promote", "pawn", "king", ("edge", "forward"), "mover")
    assert g["forward"] == {"P1": "up", "P2": "down"}
