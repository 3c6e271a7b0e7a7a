"""GAVEL-like evaluation of a game (App. F) from UCT agent-vs-agent matches.

App. F scores a (generated) game by playing matches between MCTS/UCB1 agents
(100 matches, 100 iterations per move; strategic depth against a 50-iteration
agent) and computing six heuristics, whose harmonic mean is the "GAVEL
score" (a game above 0.4 counts as potentially interesting):

* balance: one minus the gap between the two seats' win rates, so 1 is a
  perfectly balanced game (App. F lists the "max winrate gap between
  players"; as a score where higher is better it enters as 1 - gap);
* decisiveness: the fraction of matches that do not end in a draw;
* completion: the fraction of matches that reach a terminal state (a match
  that hits the game's ply cap does not);
* agency: the fraction of turns with more than one legal action;
* coverage: the fraction of the board's cells occupied at some point of a
  match, averaged over matches;
* strategic depth: the stronger agent's win rate minus the weaker agent's,
  over matches where each agent plays each seat half of the time.

The matches run on the GPU (``ludax_mcts_play``: one thread per match, the
whole match including both agents' searches in one launch); this module only
reduces the per-match counts.  A heuristic at or below zero makes the
harmonic mean zero.
"""
from __future__ import annotations

import dataclasses
import math
import time

import numpy as np

from . import dsl

HEURISTICS = ("balance", "decisiveness", "completion", "agency", "coverage", "strategic_depth")


@dataclasses.dataclass
class Matches:
    """Per-match results of one batch (numpy arrays, one entry per match)."""
    outcome: np.ndarray    # 0 draw, 1 P1 won, 2 P2 won, 3 capped (not completed)
    plies: np.ndarray
    agency: np.ndarray     # turns with more than one legal action
    coverage: np.ndarray   # cells occupied at some point
    cells: int


def harmonic_mean(values) -> float:
    v = [float(x) for x in values]
    if any(x <= 0.0 for x in v):
        return 0.0
    return len(v) / sum(1.0 / x for x in v)


def heuristics(selfplay: Matches, strong_as_p1: Matches, strong_as_p2: Matches) -> dict:
    """The six heuristics and the GAVEL score from three batches of matches:
    equal agents, the stronger agent as P1, the stronger agent as P2."""
    o = selfplay.outcome
    n = len(o)
    w1, w2 = float((o == 1).sum()) / n, float((o == 2).sum()) / n
    out = {
        "balance": 1.0 - abs(w1 - w2),
        "decisiveness": float(((o == 1) | (o == 2)).sum()) / n,
        "completion": float((o != 3).sum()) / n,
        "agency": float(selfplay.agency.astype(np.int64).sum()) / max(1, int(selfplay.plies.astype(np.int64).sum())),
        "coverage": float((selfplay.coverage.astype(np.float64) / selfplay.cells).mean()),
    }
    a, b = strong_as_p1.outcome, strong_as_p2.outcome
    m = len(a) + len(b)
    strong = int((a == 1).sum() + (b == 2).sum())
    weak = int((a == 2).sum() + (b == 1).sum())
    out["strategic_depth"] = (strong - weak) / m
    out["gavel_score"] = harmonic_mean([max(0.0, min(1.0, out[k])) for k in HEURISTICS])
    out["interesting"] = out["gavel_score"] > 0.4
    return out


def play(spec: dsl.GameSpec, matches: int, iters_p1: int, iters_p2: int, seed: int, c: float = math.sqrt(2.0),
         env_offset: int = 0) -> Matches:
    """One batch of matches of one game between UCT agents on the GPU."""
    env = dsl.make_env(spec, matches, env_offset=env_offset)
    try:
        out, plies, agency, cov = env.mcts_play(seed, iters_p1, iters_p2, c)
        res = Matches(out.cpu().numpy(), plies.cpu().numpy(), agency.cpu().numpy(), cov.cpu().numpy(), env.cells)
    finally:
        env.close()
    return res


def cells_of(spec: dsl.GameSpec) -> int:
    return 61 if spec.game == dsl.GAME_YAVALATH else spec.rows * spec.cols


def evaluate_many(games, matches: int = 100, iters: int = 100, weak_iters: int = 50, seed: int = 0,
                  c: float = math.sqrt(2.0)) -> dict:
    """Evaluate several games in ONE launch (``ludax_mcts_play_mixed``, one
    warp per match).  Game g's matches take consecutive global match
    indices: first ``matches`` between equal agents, then ``matches // 2``
    with the stronger agent as P1, then the rest with it as P2.  ``games``
    maps names to descriptions (text or compiled spec); returns {name:
    heuristics and details} plus "_seconds" (wall time of the launch)."""
    import torch

    from . import ludax

    results, parts, desc, iters_pp = {}, [], [], []
    half = max(1, matches // 2)
    sizes = ((matches, iters, iters), (half, iters, weak_iters), (max(1, matches - half), weak_iters, iters))
    for name, game in games.items():
        try:
            spec = game if isinstance(game, dsl.GameSpec) else dsl.compile_game(game)
        except dsl.DslError as err:
            results[name] = {"playable": False, "error": str(err), "gavel_score": 0.0, "interesting": False}
            continue
        spans = []
        for n, i1, i2 in sizes:
            spans.append((len(desc), n))
            desc += [spec.desc] * n
            iters_pp += [(i1, i2)] * n
        parts.append((name, spec, spans))
    n = len(desc)
    if n == 0:
        results["_seconds"] = 0.0
        return results
    dev = torch.device("cuda", torch.cuda.current_device())
    out = torch.empty(n, dtype=torch.int8, device=dev)
    plies, agency, cov = (torch.empty(n, dtype=torch.int16, device=dev) for _ in range(3))
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    ludax.ludax_mcts_play_mixed(np.array(desc, np.int32), np.array(iters_pp, np.int32), 0, seed, c, out, plies, agency,
                                cov)
    torch.cuda.synchronize()
    seconds = time.perf_counter() - t0
    o, p, a, v = (t.cpu().numpy() for t in (out, plies, agency, cov))
    for name, spec, spans in parts:
        ms = [Matches(o[s:s + k], p[s:s + k], a[s:s + k], v[s:s + k], cells_of(spec)) for s, k in spans]
        res = heuristics(*ms)
        res.update({"playable": True, "game": spec.name, "descriptor": spec.desc, "matches": matches, "iters": iters,
                    "weak_iters": weak_iters, "mean_plies": float(ms[0].plies.mean()),
                    "searches": int(sum(int(m.agency.astype(np.int64).sum()) for m in ms)),
                    "first_match": spans[0][0]})
        results[name] = res
    results["_seconds"] = seconds
    return results


def evaluate(game, matches: int = 100, iters: int = 100, weak_iters: int = 50, seed: int = 0,
             c: float = math.sqrt(2.0)) -> dict:
    """Evaluate one game description (text or compiled spec) as App. F does.
    A description that does not compile is not playable and scores 0."""
    res = evaluate_many({"game": game}, matches, iters, weak_iters, seed, c)
    out = res["game"]
    out["seconds"] = res["_seconds"]
    return out
