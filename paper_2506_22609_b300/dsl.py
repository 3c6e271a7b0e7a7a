"""Ludax game descriptions -> per-env game descriptors (Sec. 3, Sec. 4, App. B).

The paper's compiler turns each node of a game's parse tree into a JAX
closure and composes the closures bottom-up (Sec. 4).  Here the same parse
tree is lowered to DATA: a 32-bit descriptor ``game | rows << 8 | cols << 16
| line << 24 | flags << 28`` that selects one of the batched CUDA game kernels
and its parameters.  The mixed-game playout kernel and the env API consume
those descriptors directly, so a batch may hold any mix of compiled games.

Pipeline:

1. ``read`` -- S-expression reader for the grammar's surface syntax
   (App. B): parentheses, double-quoted names, integers, symbols, keyword
   arguments written ``name:`` (with or without a space before the value),
   and ``//`` comments.
2. ``elaborate`` -- a recursive descent that follows the grammar's
   productions (game, players, equipment, rules, start, play phases,
   place, effects, masks, functions, predicates, end rules, results) and
   builds a normalised intermediate form: nested tuples, ``and``/``or``
   flattened and their operands sorted, a bare function used as a
   predicate rewritten to ``(>= f 1)`` (App. B, predicate_function),
   ``(opponent win)`` rewritten to ``(mover lose)`` and vice versa.
   The move mechanics (``move`` with ``hop`` / ``slide`` / ``step``,
   priorities, ``promote``, ``extra_turn``) are elaborated like the
   placement rules.  Productions of the grammar that no kernel family
   implements (``pattern``, ``region`` / ``regions``, ``prev_move``,
   ``hopped``, ``captured``, ``promoted``, the edge and corner masks, ...)
   are recognised and rejected with the path of the offending node.
3. ``lower`` -- matches the normalised game against the kernel families
   (the m,n,k line family with exact / gravity / misere end rules, Reversi,
   Hex, Yavalath, Pente, and the move games Wolf and Sheep, English
   Draughts and Dai Hasami Shogi) and returns a ``GameSpec``.  Like the paper's
   parse-time precomputation (Sec. 4), everything that depends only on the
   description (board size, line length, rule variant) is fixed here and
   passed to the kernels as constants.  With ``specialize=True`` a line game
   that has a dedicated kernel (Tic-Tac-Toe, Connect Four, Gomoku) is mapped
   to it; otherwise to the parametric line-game kernel.

Readings of the grammar that the paper leaves open (each is a choice made
here, not a statement of the paper):

* ``(rectangle a b)`` and ``(hex_rectangle a b)`` are rows then columns.
* ``(adjacent M direction: d)`` is the set of cells reached by one step in
  direction d from a cell of M; so "the cell above an occupied cell" is
  ``(adjacent (occupied) direction: up)``.
* A ``line`` or ``connected`` without ``player:`` / ``mover:`` counts the
  mover's pieces; ``orientation`` defaults to ``any``.
* ``(custodial P n)`` is the set of opponent pieces in a run of exactly n
  (``any``: one or more) flanked on both ends by the mover's pieces, along
  the orientations given (default ``any``); as a ``result`` constraint it is
  evaluated on the position after the placement.
* ``(hexagon d)`` is the regular hexagon of diameter d; lines on it run
  along its three axes.
"""
from __future__ import annotations

import dataclasses
import os
import re

from . import ludax as _ludax

__all__ = [
    "DslError", "Sym", "Kw", "Str", "read", "elaborate", "lower", "compile_game", "compile_file",
    "descriptor", "make_env", "GameSpec", "GAMES_DIR", "library",
]

GAMES_DIR = os.path.join(os.path.dirname(os.path.abspath(__file__)), "games")

LINE_EXACT, LINE_GRAVITY, LINE_MISERE = _ludax.LUDAX_LINE_EXACT, _ludax.LUDAX_LINE_GRAVITY, _ludax.LUDAX_LINE_MISERE
GAME_TTT, GAME_C4, GAME_OTHELLO, GAME_HEX = (_ludax.LUDAX_GAME_TTT, _ludax.LUDAX_GAME_C4, _ludax.LUDAX_GAME_OTHELLO,
                                             _ludax.LUDAX_GAME_HEX)
GAME_GOMOKU, GAME_PENTE, GAME_YAVALATH, GAME_LINE = (_ludax.LUDAX_GAME_GOMOKU, _ludax.LUDAX_GAME_PENTE,
                                                     _ludax.LUDAX_GAME_YAVALATH, _ludax.LUDAX_GAME_LINE)
GAME_WOLF_SHEEP, GAME_DRAUGHTS, GAME_HASAMI_SHOGI = (_ludax.LUDAX_GAME_WOLF_SHEEP, _ludax.LUDAX_GAME_DRAUGHTS,
                                                     _ludax.LUDAX_GAME_HASAMI_SHOGI)
GAME_NAMES = {v: k for k, v in _ludax.GAME_IDS.items()}
LINE_MAX_PADDED_CELLS = 128     # rows * (cols + 1) of the parametric line-game kernel
LINE_MAX_LENGTH = 15            # four bits of the descriptor


class DslError(ValueError):
    """A description that does not parse, breaks the grammar, or uses rules
    that no kernel family implements.  ``path`` names the offending node."""

    def __init__(self, msg: str, path: str = ""):
        self.path = path
        super().__init__(f"{path}: {msg}" if path else msg)


# ------------------------------------------------------------------ reader --
@dataclasses.dataclass(frozen=True)
class Sym:
    name: str


@dataclasses.dataclass(frozen=True)
class Str:
    text: str


@dataclasses.dataclass(frozen=True)
class Kw:
    name: str


_TOKEN = re.compile(r'\s+|//[^\n]*|\(|\)|"[^"\n]*"|[^\s()"]+')


def read(text: str):
    """Parse the surface syntax into nested Python lists of Sym / Str / Kw /
    int leaves.  Exactly one top-level form is allowed."""
    toks: list[tuple[str, int]] = []
    pos, line = 0, 1
    while pos < len(text):
        m = _TOKEN.match(text, pos)
        if m is None:
            raise DslError(f"unexpected character {text[pos]!r}", f"line {line}")
        t = m.group(0)
        if not t.isspace() and not t.startswith("//"):
            if t[0] not in '()"' and ":" in t:
                # keyword argument, possibly glued to its value (exact:true)
                k, _, rest = t.partition(":")
                if not k:
                    raise DslError(f"bad keyword {t!r}", f"line {line}")
                toks.append((k + ":", line))
                if rest:
                    toks.append((rest, line))
            else:
                toks.append((t, line))
        line += t.count("\n")
        pos = m.end()

    def atom(t):
        if t.startswith('"'):
            return Str(t[1:-1])
        if t.endswith(":"):
            return Kw(t[:-1])
        if re.fullmatch(r"-?[0-9]+", t):
            return int(t)
        return Sym(t)

    stack: list[list] = [[]]
    lines: list[int] = []
    for t, ln in toks:
        if t == "(":
            stack.append([])
            lines.append(ln)
        elif t == ")":
            if len(stack) == 1:
                raise DslError("unbalanced ')'", f"line {ln}")
            done = stack.pop()
            lines.pop()
            stack[-1].append(done)
        else:
            stack[-1].append(atom(t))
    if len(stack) != 1:
        raise DslError("unclosed '('", f"line {lines[-1]}")
    if len(stack[0]) != 1:
        raise DslError(f"expected one top-level form, found {len(stack[0])}")
    return stack[0][0]


# -------------------------------------------------------------- elaborate --
def _fmt(node) -> str:
    if isinstance(node, list):
        return "(" + " ".join(_fmt(x) for x in node) + ")"
    if isinstance(node, Sym):
        return node.name
    if isinstance(node, Str):
        return f'"{node.text}"'
    if isinstance(node, Kw):
        return node.name + ":"
    return str(node)


def _head(node):
    return node[0].name if isinstance(node, list) and node and isinstance(node[0], Sym) else None


# productions of the grammar that exist but that no kernel family implements
_GRAMMAR_ONLY = {
    "pattern", "region", "regions", "prev_move", "hopped", "captured", "promoted", "edgesNoCorners", "corners",
    "edges",
}
MOVE_TYPES = ("hop", "slide", "step")

PLAYERS = ("P1", "P2")
MOVERS = ("mover", "opponent")
ORIENTATIONS = ("vertical", "horizontal", "orthogonal", "diagonal", "back_diagonal", "forward_diagonal", "any")
DIRECTIONS = ("up", "down", "left", "right", "up_left", "up_right", "down_left", "down_right", "vertical",
              "horizontal", "orthogonal", "diagonal", "back_diagonal", "forward_diagonal", "any", "forward",
              "backward", "forward_left", "forward_right", "backward_left", "backward_right")
EDGES = ("top", "bottom", "left", "right", "top_left", "top_right", "bottom_left", "bottom_right", "forward",
         "backward")


class _Elab:
    """Grammar-directed recursive descent producing the normalised form."""

    def __init__(self):
        self.pieces: dict[str, str] = {}

    # ---- helpers
    def err(self, path, msg):
        raise DslError(msg, path)

    def unsupported(self, path, node):
        self.err(path, f"'{_head(node)}' is part of the Ludax grammar but no kernel family implements it: {_fmt(node)}")

    def split(self, node, path, nmin=0):
        """Split a form's operands into positionals and keyword arguments."""
        pos, kw = [], {}
        i = 1
        while i < len(node):
            x = node[i]
            if isinstance(x, Kw):
                if i + 1 >= len(node):
                    self.err(path, f"keyword {x.name}: has no value")
                if x.name in kw:
                    self.err(path, f"keyword {x.name}: given twice")
                kw[x.name] = node[i + 1]
                i += 2
            else:
                pos.append(x)
                i += 1
        if len(pos) < nmin:
            self.err(path, f"'{_head(node)}' needs {nmin} argument(s): {_fmt(node)}")
        return pos, kw

    def expect_form(self, node, path, *names):
        h = _head(node)
        if h is None or (names and h not in names):
            want = " or ".join(f"({n} ...)" for n in names) if names else "a form"
            self.err(path, f"expected {want}, found {_fmt(node)}")
        return h

    def sym(self, x, path, allowed):
        if not isinstance(x, Sym) or x.name not in allowed:
            self.err(path, f"expected one of {', '.join(allowed)}, found {_fmt(x)}")
        return x.name

    def integer(self, x, path, lo=0):
        if not isinstance(x, int) or isinstance(x, bool) or x < lo:
            self.err(path, f"expected an integer >= {lo}, found {_fmt(x)}")
        return x

    def boolean(self, x, path):
        return self.sym(x, path, ("true", "false")) == "true"

    def piece(self, x, path):
        if not isinstance(x, Str):
            self.err(path, f"expected a piece name in double quotes, found {_fmt(x)}")
        if x.text not in self.pieces:
            self.err(path, f"piece \"{x.text}\" is not declared in (pieces ...)")
        return x.text

    def no_extra(self, kw, path, allowed):
        for k in kw:
            if k not in allowed:
                self.err(path, f"unknown keyword {k}: (allowed: {', '.join(allowed) or 'none'})")

    @staticmethod
    def assoc(op, items):
        flat = []
        for it in items:
            flat.extend(it[1] if it[0] == op else (it,))
        uniq = sorted(set(flat), key=repr)
        return uniq[0] if len(uniq) == 1 else (op, tuple(uniq))

    # ---- game
    def game(self, node):
        path = "game"
        self.expect_form(node, path, "game")
        if len(node) < 5 or not isinstance(node[1], Str):
            self.err(path, "expected (game \"name\" (players ...) (equipment ...) (rules ...) (rendering ...)?)")
        name = node[1].text
        players = self.players(node[2], path + "/players")
        board, pieces = self.equipment(node[3], path + "/equipment")
        rules = self.rules(node[4], path + "/rules")
        if len(node) > 6:
            self.err(path, f"unexpected form after (rules ...): {_fmt(node[6])}")
        if len(node) == 6:
            self.expect_form(node[5], path + "/rendering", "rendering")
        return {"name": name, "players": players, "forward": dict(self.forward), "board": board, "pieces": pieces,
                **rules}

    def players(self, node, path):
        self.expect_form(node, path, "players")
        if len(node) not in (2, 3):
            self.err(path, "expected (players n (set_forward ...)?)")
        n = self.integer(node[1], path, 1)
        self.forward = {"P1": "up", "P2": "down"}  # reading: P1 starts at the bottom
        if len(node) == 3:
            fw = node[2]
            self.expect_form(fw, path + "/set_forward", "set_forward")
            if len(fw) != 3:
                self.err(path + "/set_forward", "expected (set_forward (P1 dir) (P2 dir))")
            for who, a in zip(PLAYERS, fw[1:]):
                if not (isinstance(a, list) and len(a) == 2 and a[0] == Sym(who)):
                    self.err(path + "/set_forward", f"expected ({who} up|down|left|right), found {_fmt(a)}")
                self.forward[who] = self.sym(a[1], path + "/set_forward", ("up", "down", "left", "right"))
        return n

    def equipment(self, node, path):
        self.expect_form(node, path, "equipment")
        if len(node) not in (3, 4):
            self.err(path, "expected (equipment (board ...) (pieces ...) (regions ...)?)")
        board = self.board(node[1], path + "/board")
        self.pieces_(node[2], path + "/pieces")
        if len(node) == 4:
            self.expect_form(node[3], path + "/regions", "regions")
            self.unsupported(path + "/regions", node[3])
        return board, dict(self.pieces)

    def board(self, node, path):
        self.expect_form(node, path, "board")
        if len(node) != 2:
            self.err(path, "expected (board <shape>)")
        return self.shape(node[1], path)

    def shape(self, node, path):
        h = self.expect_form(node, path, "square", "rectangle", "hexagon", "hex_rectangle")
        pos, kw = self.split(node, path)
        self.no_extra(kw, path, ())
        want = 1 if h in ("square", "hexagon") else 2
        if len(pos) != want:
            self.err(path, f"({h} ...) takes {want} size(s)")
        dims = tuple(self.integer(x, path, 1) for x in pos)
        if h == "hexagon" and dims[0] % 2 == 0:
            self.err(path, "(hexagon d) needs an odd diameter")
        return (h,) + dims

    def pieces_(self, node, path):
        self.expect_form(node, path, "pieces")
        if len(node) < 2:
            self.err(path, "(pieces ...) declares no piece")
        for d in node[1:]:
            if not (isinstance(d, list) and len(d) == 2 and isinstance(d[0], Str)):
                self.err(path, f"expected (\"name\" P1|P2|both), found {_fmt(d)}")
            owner = self.sym(d[1], path, ("P1", "P2", "both"))
            if d[0].text in self.pieces:
                self.err(path, f"piece \"{d[0].text}\" declared twice")
            self.pieces[d[0].text] = owner

    # ---- rules
    def rules(self, node, path):
        self.expect_form(node, path, "rules")
        parts = node[1:]
        start = ()
        if parts and _head(parts[0]) == "start":
            start = self.start(parts[0], path + "/start")
            parts = parts[1:]
        if len(parts) != 2:
            self.err(path, "expected (rules (start ...)? (play ...) (end ...))")
        play = self.play(parts[0], path + "/play")
        end = self.end(parts[1], path + "/end")
        return {"start": start, "play": play, "end": end}

    def start(self, node, path):
        self.expect_form(node, path, "start")
        out = []
        for i, r in enumerate(node[1:]):
            p = f"{path}/place[{i}]"
            self.expect_form(r, p, "place")
            if len(r) != 4:
                self.err(p, "expected (place \"piece\" P1|P2 (cell ...))")
            piece = self.piece(r[1], p)
            who = self.sym(r[2], p, PLAYERS)
            if not isinstance(r[3], list) or not r[3] or not all(isinstance(c, int) for c in r[3]):
                self.err(p, f"expected a list of cell indices, found {_fmt(r[3])}")
            out.append((piece, who, tuple(sorted(self.integer(c, p) for c in r[3]))))
        if not out:
            self.err(path, "(start ...) places nothing")
        return tuple(sorted(out))

    def play(self, node, path):
        self.expect_form(node, path, "play")
        if len(node) < 2:
            self.err(path, "(play ...) has no phase")
        return tuple(self.phase(ph, f"{path}/phase[{i}]") for i, ph in enumerate(node[1:]))

    def phase(self, node, path):
        kind = self.expect_form(node, path, "once_through", "repeat")
        if len(node) not in (3, 4):
            self.err(path, f"expected ({kind} (players ...) <mechanic> (force_pass)?)")
        order = node[1]
        if not isinstance(order, list) or not order:
            self.err(path, f"expected a mover order such as (P1 P2), found {_fmt(order)}")
        order = tuple(self.sym(x, path, PLAYERS) for x in order)
        mech = self.mechanic(node[2], path + "/" + str(_head(node[2])))
        force_pass = False
        if len(node) == 4:
            self.expect_form(node[3], path, "force_pass")
            if len(node[3]) != 1:
                self.err(path, "(force_pass) takes no argument")
            force_pass = True
        return (kind, order, mech, force_pass)

    def mechanic(self, node, path):
        h = self.expect_form(node, path, "place", "move")
        if h == "move":
            return self.move(node, path)
        if len(node) < 3:
            self.err(path, "expected (place \"piece\" mover? (destination ...) (result ...)? (effects ...)?)")
        piece = self.piece(node[1], path)
        rest = node[2:]
        mover = "mover"
        if rest and isinstance(rest[0], Sym):
            mover = self.sym(rest[0], path, MOVERS)
            rest = rest[1:]
        if not rest:
            self.err(path, "(place ...) needs a (destination ...)")
        self.expect_form(rest[0], path + "/destination", "destination")
        if len(rest[0]) != 2:
            self.err(path + "/destination", "expected (destination <mask>)")
        dest = self.mask(rest[0][1], path + "/destination")
        rest = rest[1:]
        result = None
        if rest and _head(rest[0]) == "result":
            if len(rest[0]) != 2:
                self.err(path + "/result", "expected (result <predicate>)")
            result = self.pred(rest[0][1], path + "/result")
            rest = rest[1:]
        effects = ()
        if rest and _head(rest[0]) == "effects":
            if len(rest[0]) < 2:
                self.err(path + "/effects", "(effects ...) is empty")
            effects = tuple(self.effect(e, f"{path}/effects[{i}]") for i, e in enumerate(rest[0][1:]))
            rest = rest[1:]
        if rest:
            self.err(path, f"unexpected {_fmt(rest[0])}")
        return ("place", piece, mover, dest, result, effects)

    def move(self, node, path):
        if len(node) not in (2, 3):
            self.err(path, "expected (move <hop|slide|step or (or ...)> (effects ...)?)")
        spec = node[1]
        forms = spec[1:] if _head(spec) == "or" else [spec]
        if not forms:
            self.err(path, "(or) needs move types")
        types = tuple(sorted((self.move_type(f, f"{path}/{_head(f)}") for f in forms), key=repr))
        effects = ()
        if len(node) == 3:
            self.expect_form(node[2], path + "/effects", "effects")
            if len(node[2]) < 2:
                self.err(path + "/effects", "(effects ...) is empty")
            effects = tuple(self.effect(e, f"{path}/effects[{i}]") for i, e in enumerate(node[2][1:]))
        return ("move", types, effects)

    def move_type(self, node, path):
        h = self.expect_form(node, path, *MOVE_TYPES)
        pos, kw = self.split(node, path, 1)
        if len(pos) != 1:
            self.err(path, f"({h} \"piece\" ...) takes one piece")
        piece = self.piece(pos[0], path)
        dirs = self.directions(kw.get("direction"), path)
        prio = self.integer(kw["priority"], path) if "priority" in kw else 0
        if h == "hop":
            self.no_extra(kw, path, ("direction", "piece", "hop_over", "capture", "priority"))
            over = self.sym(kw["hop_over"], path, PLAYERS + MOVERS) if "hop_over" in kw else "any"
            cap = self.boolean(kw["capture"], path) if "capture" in kw else False
            target = self.piece(kw["piece"], path) if "piece" in kw else None
            return ("hop", piece, dirs, target, over, cap, prio)
        if h == "slide":
            self.no_extra(kw, path, ("direction", "distance", "priority"))
            dist = self.integer(kw["distance"], path, 1) if "distance" in kw else None
            return ("slide", piece, dirs, dist, prio)
        self.no_extra(kw, path, ("direction", "priority"))
        return ("step", piece, dirs, prio)

    # ---- effects
    def effect(self, node, path):
        h = self.expect_form(node, path)
        if h == "if":
            if len(node) == 3:
                return ("if", self.pred(node[1], path), self.effect(node[2], path + "/then"))
            if len(node) == 5 and node[3] == Sym("else"):
                return ("if", self.pred(node[1], path), self.effect(node[2], path + "/then"),
                        self.effect(node[4], path + "/else"))
            self.err(path, "expected (if <predicate> <effect>) or (if <predicate> <effect> else <effect>)")
        if h in ("flip", "capture"):
            pos, kw = self.split(node, path, 1)
            self.no_extra(kw, path, ("mover", "increment_score") if h == "capture" else ("mover",))
            if len(pos) != 1:
                self.err(path, f"({h} <mask> ...) takes one mask")
            m = self.mask(pos[0], path)
            who = self.sym(kw["mover"], path, MOVERS + ("both",)) if "mover" in kw else "mover"
            if h == "flip":
                return ("flip", m, who)
            inc = self.boolean(kw["increment_score"], path) if "increment_score" in kw else False
            return ("capture", m, who, inc)
        if h in ("set_score", "increment_score"):
            if len(node) != 3:
                self.err(path, f"expected ({h} mover|opponent <function>)")
            return (h, self.sym(node[1], path, MOVERS), self.function(node[2], path))
        if h == "promote":
            pos, kw = self.split(node, path, 3)
            self.no_extra(kw, path, ("mover",))
            if len(pos) != 3:
                self.err(path, "expected (promote \"from\" \"to\" <mask> mover: ...)")
            who = self.sym(kw["mover"], path, MOVERS + ("both",)) if "mover" in kw else "mover"
            return ("promote", self.piece(pos[0], path), self.piece(pos[1], path), self.mask(pos[2], path), who)
        if h == "extra_turn":
            pos, kw = self.split(node, path, 1)
            self.no_extra(kw, path, ("same_piece",))
            if len(pos) != 1:
                self.err(path, "expected (extra_turn mover|opponent same_piece: ...)")
            same = self.boolean(kw["same_piece"], path) if "same_piece" in kw else False
            return ("extra_turn", self.sym(pos[0], path, MOVERS), same)
        if h in _GRAMMAR_ONLY:
            self.unsupported(path, node)
        self.err(path, f"unknown effect {_fmt(node)}")

    # ---- masks
    def mask(self, node, path):
        h = self.expect_form(node, path)
        if h in ("and", "or"):
            if len(node) < 2:
                self.err(path, f"({h}) needs operands")
            return self.assoc(h, [self.mask(x, f"{path}/{h}[{i}]") for i, x in enumerate(node[1:])])
        if h == "not":
            if len(node) != 2:
                self.err(path, "expected (not <mask>)")
            inner = self.mask(node[1], path + "/not")
            return inner[1] if inner[0] == "not" else ("not", inner)
        if h in ("empty", "center", "corners"):
            if len(node) != 1:
                self.err(path, f"({h}) takes no argument")
            if h == "corners":
                self.unsupported(path, node)
            return (h,)
        if h == "occupied":
            if len(node) > 2:
                self.err(path, "expected (occupied mover|opponent?)")
            return ("occupied", self.sym(node[1], path, MOVERS) if len(node) == 2 else "any")
        if h in ("row", "column"):
            if len(node) != 2:
                self.err(path, f"expected ({h} n)")
            return (h, self.integer(node[1], path))
        if h == "edge":
            if len(node) != 2:
                self.err(path, "expected (edge <side>)")
            return ("edge", self.sym(node[1], path, EDGES))
        if h == "adjacent":
            pos, kw = self.split(node, path, 1)
            self.no_extra(kw, path, ("direction",))
            if len(pos) != 1:
                self.err(path, "expected (adjacent <mask> direction: d?)")
            return ("adjacent", self.mask(pos[0], path + "/adjacent"), self.directions(kw.get("direction"), path))
        if h == "custodial":
            pos, kw = self.split(node, path, 2)
            self.no_extra(kw, path, ("mover", "orientation"))
            if len(pos) != 2:
                self.err(path, "expected (custodial \"piece\" n|any mover: ... orientation: ...)")
            piece = self.piece(pos[0], path)
            n = "any" if pos[1] == Sym("any") else self.integer(pos[1], path, 1)
            who = self.sym(kw["mover"], path, MOVERS + ("both",)) if "mover" in kw else "mover"
            orient = self.sym(kw["orientation"], path, ORIENTATIONS) if "orientation" in kw else "any"
            return ("custodial", piece, n, who, orient)
        if h == "corner_custodial":
            pos, kw = self.split(node, path, 1)
            self.no_extra(kw, path, ("mover",))
            if len(pos) != 1:
                self.err(path, "expected (corner_custodial \"piece\" mover: ...)")
            who = self.sym(kw["mover"], path, MOVERS + ("both",)) if "mover" in kw else "mover"
            return ("corner_custodial", self.piece(pos[0], path), who)
        if h == "line":
            self.err(path, f"(line ...) as a mask of cells is not implemented by any kernel family: {_fmt(node)}")
        if h in _GRAMMAR_ONLY:
            self.unsupported(path, node)
        self.err(path, f"unknown mask {_fmt(node)}")

    def directions(self, x, path):
        if x is None:
            return ("any",)
        if isinstance(x, list):
            if not x:
                self.err(path, "empty direction list")
            return tuple(sorted({self.sym(d, path, DIRECTIONS) for d in x}))
        return (self.sym(x, path, DIRECTIONS),)

    # ---- functions
    def function(self, node, path):
        if isinstance(node, int) and not isinstance(node, bool):
            return ("const", self.integer(node, path))
        h = self.expect_form(node, path)
        if h == "line":
            pos, kw = self.split(node, path, 2)
            self.no_extra(kw, path, ("orientation", "exact", "player", "exclude"))
            if len(pos) != 2:
                self.err(path, "expected (line \"piece\" n ...)")
            piece = self.piece(pos[0], path)
            n = self.integer(pos[1], path, 1)
            orient = self.sym(kw["orientation"], path, ORIENTATIONS) if "orientation" in kw else "any"
            exact = self.boolean(kw["exact"], path) if "exact" in kw else False
            who = self.sym(kw["player"], path, PLAYERS + MOVERS) if "player" in kw else "mover"
            excl = self.multi_mask(kw["exclude"], path + "/exclude") if "exclude" in kw else ()
            return ("line", piece, n, orient, exact, who, excl)
        if h == "connected":
            pos, kw = self.split(node, path, 2)
            self.no_extra(kw, path, ("mover", "direction"))
            if len(pos) != 2:
                self.err(path, "expected (connected \"piece\" (<mask> <mask> ...) ...)")
            piece = self.piece(pos[0], path)
            masks = self.multi_mask(pos[1], path + "/connected")
            who = self.sym(kw["mover"], path, MOVERS + ("both",)) if "mover" in kw else "mover"
            return ("connected", piece, masks, who, self.directions(kw.get("direction"), path))
        if h == "count":
            if len(node) != 2:
                self.err(path, "expected (count <mask>)")
            return ("count", self.mask(node[1], path + "/count"))
        if h == "score":
            if len(node) != 2:
                self.err(path, "expected (score mover|opponent)")
            return ("score", self.sym(node[1], path, MOVERS))
        if h in ("add", "multiply"):
            if len(node) < 2:
                self.err(path, f"({h}) needs operands")
            return (h, tuple(sorted((self.function(x, path) for x in node[1:]), key=repr)))
        if h == "subtract":
            if len(node) != 3:
                self.err(path, "expected (subtract f g)")
            return ("subtract", self.function(node[1], path), self.function(node[2], path))
        if h in _GRAMMAR_ONLY:
            self.unsupported(path, node)
        self.err(path, f"unknown function {_fmt(node)}")

    def multi_mask(self, x, path):
        if isinstance(x, list) and x and isinstance(x[0], list):
            return tuple(sorted((self.mask(m, path) for m in x), key=repr))
        h = _head(x)
        if h in ("corners", "edges", "edgesNoCorners"):
            self.unsupported(path, x)
        return (self.mask(x, path),)

    # ---- predicates
    _FUNCS = ("line", "connected", "count", "score", "add", "multiply", "subtract")

    def pred(self, node, path):
        if isinstance(node, int):
            return ("ge", ("const", node), ("const", 1))
        h = self.expect_form(node, path)
        if h in ("and", "or"):
            if len(node) < 2:
                self.err(path, f"({h}) needs operands")
            return self.assoc(h, [self.pred(x, f"{path}/{h}[{i}]") for i, x in enumerate(node[1:])])
        if h == "not":
            if len(node) != 2:
                self.err(path, "expected (not <predicate>)")
            inner = self.pred(node[1], path + "/not")
            return inner[1] if inner[0] == "not" else ("not", inner)
        if h in ("full_board", "no_legal_actions"):
            if len(node) != 1:
                self.err(path, f"({h}) takes no argument")
            return (h,)
        if h == "passed":
            if len(node) != 2:
                self.err(path, "expected (passed mover|opponent|both)")
            return ("passed", self.sym(node[1], path, MOVERS + ("both",)))
        if h == "mover_is":
            if len(node) != 2:
                self.err(path, "expected (mover_is P1|P2)")
            return ("mover_is", self.sym(node[1], path, PLAYERS))
        if h == "last_move_in":
            if len(node) != 2:
                self.err(path, "expected (last_move_in <mask>)")
            return ("last_move_in", self.mask(node[1], path + "/last_move_in"))
        if h == "action_was":
            if len(node) != 3:
                self.err(path, "expected (action_was mover|opponent hop|slide|step)")
            return ("action_was", self.sym(node[1], path, MOVERS), self.sym(node[2], path, MOVE_TYPES))
        if h == "can_move_again":
            if len(node) != 2:
                self.err(path, "expected (can_move_again hop|slide|step)")
            return ("can_move_again", self.sym(node[1], path, MOVE_TYPES))
        if h == "exists":
            if len(node) != 2:
                self.err(path, "expected (exists <mask>)")
            return ("ge", ("count", self.mask(node[1], path + "/exists")), ("const", 1))
        if h in (">=", "<="):
            if len(node) != 3:
                self.err(path, f"expected ({h} f g)")
            f, g = self.function(node[1], path), self.function(node[2], path)
            return ("ge", f, g) if h == ">=" else ("ge", g, f)
        if h == "=":
            if len(node) < 3:
                self.err(path, "(= ...) needs two or more functions")
            return ("eq", tuple(sorted((self.function(x, path) for x in node[1:]), key=repr)))
        if h in self._FUNCS:
            return ("ge", self.function(node, path), ("const", 1))
        if h in _GRAMMAR_ONLY:
            self.unsupported(path, node)
        self.err(path, f"unknown predicate {_fmt(node)}")

    # ---- end rules
    def end(self, node, path):
        self.expect_form(node, path, "end")
        if len(node) < 2:
            self.err(path, "(end ...) has no rule")
        out = []
        for i, r in enumerate(node[1:]):
            p = f"{path}/if[{i}]"
            self.expect_form(r, p, "if")
            if len(r) != 3:
                self.err(p, "expected (if <predicate> <result>)")
            out.append((self.pred(r[1], p), self.result(r[2], p)))
        return tuple(out)

    def result(self, node, path):
        h = self.expect_form(node, path)
        if h == "draw" and len(node) == 1:
            return ("draw",)
        if h == "by_score" and len(node) == 1:
            return ("by_score",)
        if isinstance(node, list) and len(node) == 2 and isinstance(node[1], Sym) and node[1].name in ("win", "lose"):
            who = self.sym(node[0], path, MOVERS + ("both",))
            win = node[1].name == "win"
            if who == "opponent":       # two players: the opponent winning is the mover losing
                who, win = "mover", not win
            return ("win" if win else "lose", who)
        self.err(path, f"expected (mover|opponent|both win|lose), (draw) or (by_score), found {_fmt(node)}")


def elaborate(form) -> dict:
    """Normalised form of a parsed game (see the module docstring)."""
    return _Elab().game(form)


# ------------------------------------------------------------------ lower --
@dataclasses.dataclass(frozen=True)
class GameSpec:
    """A compiled game: the kernel family, its parameters and the descriptor."""
    name: str
    game: int          # LUDAX_GAME_* id of the kernel
    rows: int
    cols: int
    line: int = 0      # parametric line game only
    flags: int = 0     # LINE_EXACT | LINE_GRAVITY | LINE_MISERE
    desc: int = 0

    @property
    def family(self) -> str:
        return GAME_NAMES[self.game]


def _spec(name, game, rows, cols, line=0, flags=0):
    d = game | (rows << 8) | (cols << 16) | (line << 24) | (flags << 28)
    return GameSpec(name, game, rows, cols, line, flags, d)


EMPTY = ("empty",)
# cells that are empty and either on the bottom row or directly above a stone
GRAVITY = ("and", tuple(sorted([EMPTY, ("or", tuple(sorted([
    ("edge", "bottom"), ("adjacent", ("occupied", "any"), ("up",))], key=repr)))], key=repr)))
FULL_DRAW = (("full_board",), ("draw",))


def _line_pred(p):
    """(n, exact) if p is 'the mover has a line of n, any orientation'."""
    if p[0] == "ge" and p[2] == ("const", 1) and p[1][0] == "line":
        _, _piece, n, orient, exact, who, excl = p[1]
        if orient == "any" and who == "mover" and not excl:
            return n, exact
    return None


def _fail(path, msg):
    raise DslError(msg, path)


def _single_alternating_place(g, path="rules/play"):
    play = g["play"]
    if len(play) != 1:
        _fail(path, "this kernel family takes a single (repeat (P1 P2) ...) phase")
    kind, order, mech, force_pass = play[0]
    if kind != "repeat" or order != ("P1", "P2"):
        _fail(path, "players must alternate with P1 first: (repeat (P1 P2) ...)")
    if mech[2] != "mover":
        _fail(path + "/place", "pieces are placed by the mover")
    return mech, force_pass


def _lower_line(g, specialize):
    shape = g["board"]
    rows, cols = (shape[1], shape[1]) if shape[0] == "square" else (shape[1], shape[2])
    if g["start"]:
        _fail("rules/start", "line games start from the empty board")
    mech, force_pass = _single_alternating_place(g)
    _, _piece, _mover, dest, result, effects = mech
    if force_pass or result is not None or effects:
        _fail("rules/play/place", "a line game places one stone and has no result constraint, effects or passes")
    flags = 0
    if dest == GRAVITY:
        flags |= LINE_GRAVITY
    elif dest != EMPTY:
        _fail("rules/play/place/destination", "supported destinations: (empty), or (empty) on the bottom edge or "
              "above an occupied cell (gravity)")
    end = g["end"]
    if len(end) != 2 or end[1] != FULL_DRAW:
        _fail("rules/end", "a line game has exactly two end rules: a line rule, then (if (full_board) (draw))")
    lp = _line_pred(end[0][0])
    if lp is None:
        _fail("rules/end/if[0]", "the first end rule must be (line \"piece\" n) of the mover in every orientation")
    n, exact = lp
    res = end[0][1]
    if res not in (("win", "mover"), ("lose", "mover")):
        _fail("rules/end/if[0]", "a line ends the game with (mover win) or (mover lose)")
    flags |= (LINE_EXACT if exact else 0) | (LINE_MISERE if res[0] == "lose" else 0)
    if n < 2 or n > max(rows, cols):
        _fail("rules/end/if[0]", f"a line of {n} on a {rows}x{cols} board is not a playable line game")
    name = g["name"]
    if specialize:
        if (rows, cols, n, flags) == (3, 3, 3, 0):
            return _spec(name, GAME_TTT, 3, 3)
        if (rows, cols, n, flags) == (6, 7, 4, LINE_GRAVITY):
            return _spec(name, GAME_C4, 6, 7)
    if (rows, cols, n, flags) == (15, 15, 5, LINE_EXACT):
        return _spec(name, GAME_GOMOKU, 15, 15)
    if rows * (cols + 1) > LINE_MAX_PADDED_CELLS:
        _fail("equipment/board", f"{rows}x{cols} is larger than the line-game kernel's board "
              f"(rows * (cols + 1) <= {LINE_MAX_PADDED_CELLS})")
    if n > LINE_MAX_LENGTH:
        _fail("rules/end/if[0]", f"line length {n} > {LINE_MAX_LENGTH}")
    return _spec(name, GAME_LINE, rows, cols, n, flags)


def _lower_yavalath(g):
    if g["board"] != ("hexagon", 9):
        _fail("equipment/board", "the hexagon kernel implements (hexagon 9)")
    if g["start"]:
        _fail("rules/start", "Yavalath starts from the empty board")
    mech, force_pass = _single_alternating_place(g)
    if force_pass or mech[3] != EMPTY or mech[4] is not None or mech[5]:
        _fail("rules/play/place", "Yavalath places one stone on an empty cell, nothing else")
    end = g["end"]
    ok = len(end) == 3 and end[2] == FULL_DRAW
    if ok:
        a, b = _line_pred(end[0][0]), _line_pred(end[1][0])
        # "four wins" first; after it a line of three (exact or not) is exactly three
        ok = a == (4, False) and end[0][1] == ("win", "mover") and b in ((3, False), (3, True)) \
            and end[1][1] == ("lose", "mover")
    if not ok:
        _fail("rules/end", "the hexagon kernel implements: a line of 4 wins, then a line of 3 loses, "
              "then a full board draws")
    return _spec(g["name"], GAME_YAVALATH, 9, 9)


def _lower_hex(g):
    _, rows, cols = g["board"]
    if rows != cols or not 2 <= rows <= 11:
        _fail("equipment/board", "the Hex kernel implements (hex_rectangle n n), 2 <= n <= 11")
    if g["start"]:
        _fail("rules/start", "Hex starts from the empty board")
    mech, force_pass = _single_alternating_place(g)
    if force_pass or mech[3] != EMPTY or mech[4] is not None or mech[5]:
        _fail("rules/play/place", "Hex places one stone on an empty cell, nothing else")
    piece = mech[1]

    def conn(a, b):
        return ("ge", ("connected", piece, tuple(sorted([("edge", a), ("edge", b)], key=repr)), "mover", ("any",)),
                ("const", 1))

    p1 = ("and", tuple(sorted([("mover_is", "P1"), conn("top", "bottom")], key=repr)))
    p2 = ("and", tuple(sorted([("mover_is", "P2"), conn("left", "right")], key=repr)))
    win = ("win", "mover")
    end = g["end"]
    forms = [((p1, win), (p2, win)), ((p2, win), (p1, win)), ((("or", tuple(sorted([p1, p2], key=repr))), win),)]
    if tuple(end) not in forms:
        _fail("rules/end", "the Hex kernel implements: the mover wins when P1 connects (edge top) and "
              "(edge bottom), or P2 connects (edge left) and (edge right)")
    return _spec(g["name"], GAME_HEX, rows, rows)


def _lower_reversi(g):
    if g["board"] != ("square", 8):
        _fail("equipment/board", "the Reversi kernel implements (square 8)")
    mech, force_pass = _single_alternating_place(g)
    _, piece, _, dest, result, effects = mech
    if [(w, c) for (_p, w, c) in g["start"]] != [("P1", (28, 35)), ("P2", (27, 36))]:
        _fail("rules/start", "the Reversi start is P1 on cells 28 and 35, P2 on 27 and 36")
    if not force_pass:
        _fail("rules/play", "Reversi passes when no placement is legal: add (force_pass)")
    if dest != EMPTY:
        _fail("rules/play/place/destination", "Reversi places on an (empty) cell")
    flank = ("custodial", piece, "any", "mover", "any")
    if result != ("ge", ("count", flank), ("const", 1)):
        _fail("rules/play/place/result", "the placement must flank: (exists (custodial \"piece\" any))")
    scores = {("set_score", "mover", ("count", ("occupied", "mover"))),
              ("set_score", "opponent", ("count", ("occupied", "opponent")))}
    eff = set(effects)
    if len(eff) != len(effects) or ("flip", flank, "mover") not in eff or \
            eff - {("flip", flank, "mover")} not in (set(), scores):
        _fail("rules/play/place/effects", "Reversi flips (custodial \"piece\" any); scores, if set, count "
              "each player's pieces")
    if g["end"] != ((("passed", "both"), ("by_score",)),):
        _fail("rules/end", "Reversi ends when both players have passed, by score: (if (passed both) (by_score))")
    return _spec(g["name"], GAME_OTHELLO, 8, 8)


def _lower_pente(g):
    if g["board"] != ("square", 19):
        _fail("equipment/board", "the Pente kernel implements (square 19)")
    if g["start"]:
        _fail("rules/start", "Pente starts from the empty board")
    play = g["play"]
    if len(play) != 2:
        _fail("rules/play", "Pente has two phases: P1's first stone, then alternation")
    (k1, o1, m1, f1), (k2, o2, m2, f2) = play
    if k1 != "once_through" or o1 != ("P1",) or f1 or m1[2] != "mover" or m1[3] not in (
            ("center",), ("and", tuple(sorted([EMPTY, ("center",)], key=repr)))) or m1[4] is not None or m1[5]:
        _fail("rules/play/phase[0]", "Pente's first phase is (once_through (P1) (place \"piece\" (destination "
              "(center))))")
    cap = ("capture", ("custodial", m2[1], 2, "mover", "any"), "mover", True)
    if k2 != "repeat" or o2 != ("P2", "P1") or f2 or m2[2] != "mover" or m2[3] != EMPTY or m2[4] is not None \
            or m2[5] != (cap,):
        _fail("rules/play/phase[1]", "Pente's second phase alternates from P2, places on (empty) cells and "
              "captures (custodial \"piece\" 2) with increment_score: true")
    end = g["end"]
    want = [(("ge", ("line", m2[1], 5, "any", False, "mover", ()), ("const", 1)), ("win", "mover")),
            (("ge", ("score", "mover"), ("const", 10)), ("win", "mover")), FULL_DRAW]
    if len(end) != 3 or end[2] != FULL_DRAW or sorted(end[:2], key=repr) != sorted(want[:2], key=repr):
        _fail("rules/end", "the Pente kernel implements: a line of five or a score of 10 wins, then a full "
              "board draws")
    return _spec(g["name"], GAME_PENTE, 19, 19)


FWD_DIAGONALS = (("forward_left", "forward_right"),)
WIN = ("win", "mover")
NO_MOVES_WIN = (("no_legal_actions",), WIN)


def _dark_cells(rows):
    return tuple(r * 8 + c for r in rows for c in range(8) if (r + c) % 2 == 1)


def _forward_ok(g, path):
    if g["forward"] != {"P1": "up", "P2": "down"}:
        _fail(path, "the move-game kernels take P1 moving up and P2 down: (set_forward (P1 up) (P2 down))")


def _single_move_phase(g, path="rules/play"):
    play = g["play"]
    if len(play) != 1:
        _fail(path, "the move-game kernels take a single (repeat (P1 P2) (move ...)) phase")
    kind, order, mech, force_pass = play[0]
    if kind != "repeat" or order != ("P1", "P2"):
        _fail(path, "players must alternate with P1 first: (repeat (P1 P2) ...)")
    if mech[0] != "move" or force_pass:
        _fail(path, "the move-game kernels take one (move ...) mechanic and no pass")
    return mech[1], mech[2]   # move types, effects


def _lower_wolf_sheep(g):
    sheep = [k for k, v in g["pieces"].items() if v == "P1"]
    wolf = [k for k, v in g["pieces"].items() if v == "P2"]
    if len(sheep) != 1 or len(wolf) != 1 or len(g["pieces"]) != 2:
        _fail("equipment/pieces", "Wolf and Sheep has one piece type of P1 (sheep) and one of P2 (wolf)")
    a, b = sheep[0], wolf[0]
    if g["start"] != tuple(sorted([(a, "P1", (56, 58, 60, 62)), (b, "P2", (3,))])):
        _fail("rules/start", "the Wolf and Sheep kernel starts with sheep on 56 58 60 62 and the wolf on 3")
    types, effects = _single_move_phase(g)
    fwd = [("step", a, d, 0) for d in (("forward_left", "forward_right"), ("up_left", "up_right"))]
    ok = any(types == tuple(sorted([f, ("step", b, ("diagonal",), 0)], key=repr)) for f in fwd)
    if not ok or effects:
        _fail("rules/play", "Wolf and Sheep: sheep step diagonally forward, the wolf diagonally, no effects")
    bottom = (("and", tuple(sorted([("mover_is", "P2"), ("last_move_in", ("edge", "bottom"))], key=repr))), WIN)
    if tuple(g["end"]) not in ((bottom, NO_MOVES_WIN), (NO_MOVES_WIN, bottom)):
        _fail("rules/end", "Wolf and Sheep ends when the wolf reaches the bottom edge or a side cannot move")
    return _spec(g["name"], GAME_WOLF_SHEEP, 8, 8)


def _lower_draughts(g):
    if len(g["pieces"]) != 2 or set(g["pieces"].values()) != {"both"}:
        _fail("equipment/pieces", "Draughts has two piece types of both players (a man and a king)")
    types, effects = _single_move_phase(g)
    men = [t[1] for t in types if t[0] == "step" and t[2] == ("forward_left", "forward_right")]
    if len(men) != 1:
        _fail("rules/play", "Draughts: men step diagonally forward (forward_left forward_right)")
    m = men[0]
    k = [x for x in g["pieces"] if x != m][0]
    fwd, diag = ("forward_left", "forward_right"), ("diagonal",)
    want = tuple(sorted([("hop", m, fwd, None, "opponent", True, 0), ("hop", k, diag, None, "opponent", True, 0),
                         ("step", m, fwd, 1), ("step", k, diag, 1)], key=repr))
    if types != want:
        _fail("rules/play", "Draughts: hops over an opponent (capture, priority 0) before steps (priority 1), men "
              "forward, kings diagonally")
    if g["start"] != tuple(sorted([(m, "P1", _dark_cells((5, 6, 7))), (m, "P2", _dark_cells((0, 1, 2)))])):
        _fail("rules/start", "the Draughts kernel starts with men on the dark cells of rows 5-7 (P1) and 0-2 (P2)")
    again = ("and", tuple(sorted([("action_was", "mover", "hop"), ("can_move_again", "hop")], key=repr)))
    if effects != (("promote", m, k, ("edge", "forward"), "mover"), ("if", again, ("extra_turn", "mover", True))):
        _fail("rules/play/effects", "Draughts: promote men on the forward edge, then an extra turn for the same "
              "piece after a hop that can be continued")
    if tuple(g["end"]) != (NO_MOVES_WIN,):
        _fail("rules/end", "Draughts ends when the player to move has no legal action")
    return _spec(g["name"], GAME_DRAUGHTS, 8, 8)


def _lower_hasami(g):
    if len(g["pieces"]) != 1 or set(g["pieces"].values()) != {"both"}:
        _fail("equipment/pieces", "Dai Hasami Shogi uses one piece type of both players")
    p = next(iter(g["pieces"]))
    if g["start"] != tuple(sorted([(p, "P1", tuple(range(63, 81))), (p, "P2", tuple(range(0, 18)))])):
        _fail("rules/start", "the Dai Hasami Shogi kernel starts with P1 on rows 7-8 and P2 on rows 0-1")
    types, effects = _single_move_phase(g)
    orth = ("orthogonal",)
    slide = ("slide", p, orth, None, 0)
    hops = [tuple(sorted([slide, ("hop", p, orth, None, "any", False, 0)], key=repr)),
            tuple(sorted([slide, ("hop", p, orth, None, "mover", False, 0), ("hop", p, orth, None, "opponent", False, 0)],
                         key=repr))]
    if types not in hops:
        _fail("rules/play", "Dai Hasami Shogi: orthogonal slides and hops over one piece of either side (no capture)")
    caps = {("capture", ("custodial", p, "any", "mover", "orthogonal"), "mover", False),
            ("capture", ("corner_custodial", p, "mover"), "mover", False)}
    if set(effects) != caps or len(effects) != 2:
        _fail("rules/play/effects", "Dai Hasami Shogi captures custodially (any length, orthogonal) and in corners")

    def five(who, rows):
        line = ("ge", ("line", p, 5, "orthogonal", False, "mover", tuple(sorted((("row", r) for r in rows), key=repr))),
                ("const", 1))
        return (("and", tuple(sorted([("mover_is", who), line], key=repr))), WIN)

    r1, r2 = five("P1", (7, 8)), five("P2", (0, 1))
    if tuple(g["end"]) not in ((r1, r2, NO_MOVES_WIN), (r2, r1, NO_MOVES_WIN)):
        _fail("rules/end", "Dai Hasami Shogi: five in a row (orthogonal) outside the mover's home rows wins, then a "
              "side without a move loses")
    return _spec(g["name"], GAME_HASAMI_SHOGI, 9, 9)


def _lower_move_game(g):
    _forward_ok(g, "players")
    shape = g["board"]
    if shape == ("square", 9):
        return _lower_hasami(g)
    if shape != ("square", 8):
        _fail("equipment/board", "the move-game kernels take (square 8) (Wolf and Sheep, Draughts) or (square 9)")
    owners = set(g["pieces"].values())
    return _lower_draughts(g) if owners == {"both"} else _lower_wolf_sheep(g)


def lower(g: dict, specialize: bool = True) -> GameSpec:
    """Match a normalised game against the kernel families."""
    if g["players"] != 2:
        _fail("players", "every kernel family is a two-player game")
    if any(ph[2][0] == "move" for ph in g["play"]):
        return _lower_move_game(g)
    owners = set(g["pieces"].values())
    if len(g["pieces"]) != 1 or owners != {"both"}:
        _fail("equipment/pieces", "every kernel family uses one piece type shared by both players (\"name\" both)")
    shape = g["board"][0]
    if shape == "hex_rectangle":
        return _lower_hex(g)
    if shape == "hexagon":
        return _lower_yavalath(g)
    if g["start"]:
        return _lower_reversi(g)
    if len(g["play"]) == 2:
        return _lower_pente(g)
    return _lower_line(g, specialize)


def compile_game(text: str, specialize: bool = True) -> GameSpec:
    """Game description text -> compiled ``GameSpec``."""
    return lower(elaborate(read(text)), specialize)


def compile_file(path: str, specialize: bool = True) -> GameSpec:
    with open(path) as f:
        return compile_game(f.read(), specialize)


def descriptor(text: str, specialize: bool = True) -> int:
    """The int32 descriptor that the mixed-game kernel and plan consume."""
    return compile_game(text, specialize).desc


def library() -> dict[str, str]:
    """The game descriptions shipped with the package, by file stem."""
    out = {}
    for fn in sorted(os.listdir(GAMES_DIR)):
        if fn.endswith(".ldx"):
            with open(os.path.join(GAMES_DIR, fn)) as f:
                out[fn[:-4]] = f.read()
    return out


def make_env(text_or_spec, num_envs: int, **kw) -> "_ludax.Env":
    """A batched env of ``num_envs`` copies of a compiled game."""
    s = text_or_spec if isinstance(text_or_spec, GameSpec) else compile_game(text_or_spec)
    return _ludax.Env(GAME_NAMES[s.game], s.rows, s.cols, num_envs, line=s.line, flags=s.flags, **kw)
