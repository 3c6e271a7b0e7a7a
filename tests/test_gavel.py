"""GAVEL-like heuristics (App. F) from per-match counts.  CPU only."""
import numpy as np

from paper_2506_22609_b300 import gavel


def M(outcome, plies=None, agency=None, coverage=None, cells=9):
    o = np.array(outcome, np.int8)
    n = len(o)
    return gavel.Matches(o, np.array(plies if plies is not None else [9] * n, np.int16),
                         np.array(agency if agency is not None else [8] * n, np.int16),
                         np.array(coverage if coverage is not None else [9] * n, np.int16), cells)


def test_heuristics_closed_form():
    self_ = M([1, 1, 2, 0], plies=[5, 7, 6, 9], agency=[4, 6, 5, 8], coverage=[5, 7, 6, 9])
    sp1 = M([1, 1, 0, 2])       # strong as P1: 2 wins, 1 loss
    sp2 = M([2, 0, 0, 1])       # strong as P2: 1 win, 1 loss
    h = gavel.heuristics(self_, sp1, sp2)
    assert h["balance"] == 1 - abs(0.5 - 0.25)
    assert h["decisiveness"] == 0.75
    assert h["completion"] == 1.0
    assert h["agency"] == (4 + 6 + 5 + 8) / (5 + 7 + 6 + 9)
    assert abs(h["coverage"] - np.mean([5 / 9, 7 / 9, 6 / 9, 1.0])) < 1e-12
    assert h["strategic_depth"] == (3 - 2) / 8
    vals = [h[k] for k in gavel.HEURISTICS]
    assert abs(h["gavel_score"] - 6 / sum(1 / v for v in vals)) < 1e-12


def test_harmonic_mean_is_zero_when_a_heuristic_is():
    # all draws: decisiveness 0 -> score 0; capped matches are not complete
    h = gavel.heuristics(M([0, 0, 3, 3]), M([1, 1]), M([2, 2]))
    assert h["decisiveness"] == 0.0 and h["completion"] == 0.5 and h["gavel_score"] == 0.0
    assert not h["interesting"]
    # the weaker agent winning gives negative depth, clipped to 0 in the score
    h = gavel.heuristics(M([1, 2]), M([2, 2]), M([1, 1]))
    assert h["strategic_depth"] == -1.0 and h["gavel_score"] == 0.0
    assert gavel.harmonic_mean([1, 1, 1]) == 1.0 and gavel.harmonic_mean([0.5, 1.0]) == 2 / 3


def test_unplayable_description_scores_zero():
    res = gavel.evaluate("(game \"broken\" (players 2)")
    assert res["playable"] is False and res["gavel_score"] == 0.0
