"""GPU: the packed state view (two bits per cell) against the byte view and
the oracle, for every game family.

Oracle positions at random plies go in through one view and out through the
other, bit-exact; the same positions loaded through either view then play
identical playouts (the engine's derived state -- Hex edge sets, Draughts
capture caches, Hasami Shogi's transposed occupancy -- is rebuilt the same).
"""
import numpy as np
import pytest
import torch

from oracle import games as G


def pack_state_bits(board, to_move, ply, passes, outcome, planes_count):
    """Test-side encoder of the packed state (numpy, host) of a canonical
    state view: planes uint64 [planes_count * W][n] and meta uint32 [n], as
    ludax_get_state_bits writes them."""
    board = np.asarray(board)
    n, cells = board.shape
    W = (cells + 63) // 64
    planes = np.zeros((planes_count * W, n), np.uint64)
    for v in range(1, planes_count + 1):
        for c in range(cells):
            hit = (board[:, c] == v).astype(np.uint64)
            planes[(v - 1) * W + c // 64] |= hit << np.uint64(c % 64)
    meta = (np.asarray(ply).astype(np.uint32) & 0xFFFF) | ((np.asarray(to_move).astype(np.uint32) - 1) & 1) << 16 | \
        (np.asarray(passes).astype(np.uint8).astype(np.uint32) << 17) | \
        (((np.asarray(outcome).astype(np.int32) + 1) & 7).astype(np.uint32) << 25)
    return planes, meta.astype(np.uint32)


pytestmark = pytest.mark.gpu

CASES = [("ttt", G.TTT, 3, 3), ("c4", G.C4, 6, 7), ("othello", G.OTHELLO, 8, 8), ("hex5", G.HEX, 5, 5),
         ("hex11", G.HEX, 11, 11), ("gomoku", G.GOMOKU, 15, 15), ("pente", G.PENTE, 19, 19),
         ("yavalath", G.YAVALATH, 9, 9), ("wolf_sheep", G.WOLF_SHEEP, 8, 8), ("draughts", G.DRAUGHTS, 8, 8),
         ("hasami_shogi", G.HASAMI_SHOGI, 9, 9)]


@pytest.fixture(scope="module")
def L(cuda_device):
    from paper_2506_22609_b300 import build

    build.build()
    from paper_2506_22609_b300 import ludax

    ludax.lib()
    return ludax


def positions(game, rows, cols, n, seed):
    s = G.reset(game, rows, cols, n)
    cells = G.num_cells(game, rows, cols)
    rng = np.random.default_rng(seed)
    stop = rng.integers(0, max(2, cells), n).astype(np.int16)
    G.rollout_from(s, seed=seed, stop_ply=stop)
    return s


@pytest.mark.parametrize("name,game,rows,cols", CASES, ids=[c[0] for c in CASES])
def test_packed_view_round_trips(L, name, game, rows, cols):
    n = 333  # two 128-thread tiles and a ragged tail
    s = positions(game, rows, cols, n, 17)
    view = (s.board, s.to_move, s.ply, s.passes, s.outcome)
    planes_count = 4 if game == G.DRAUGHTS else 2
    want_p, want_m = pack_state_bits(*view, planes_count)

    a = L.Env(game, rows, cols, n, env_offset=5)
    a.set_state(*(torch.from_numpy(x) for x in view))
    assert a.state_bits_words() == want_p.shape[0]
    p, m = a.get_state_bits()
    torch.cuda.synchronize()
    assert (p.cpu().numpy().view(np.uint64) == want_p).all()
    assert (m.cpu().numpy().view(np.uint32) == want_m).all()

    b = L.Env(game, rows, cols, n, env_offset=5)
    b.set_state_bits(torch.from_numpy(want_p.view(np.int64)), torch.from_numpy(want_m.view(np.int32)))
    got = [t.cpu().numpy() for t in b.get_state()]
    for g_, w_ in zip(got, view):
        assert (g_ == w_).all()

    oa, pa = a.rollout(42, from_start=False)
    ob, pb = b.rollout(42, from_start=False)
    torch.cuda.synchronize()
    assert (oa.cpu().numpy() == ob.cpu().numpy()).all() and (pa.cpu().numpy() == pb.cpu().numpy()).all()
    t = s.copy()
    G.rollout_from(t, seed=42, env_offset=5)
    assert (oa.cpu().numpy() == t.outcome).all()
    for e in (a, b):
        e.close()


def test_packed_view_ignores_bits_past_the_board(L):
    n = 64
    s = positions(G.C4, 6, 7, n, 3)
    p, m = pack_state_bits(s.board, s.to_move, s.ply, s.passes, s.outcome, 2)
    junk = p.copy()
    junk |= np.uint64(0xFFFFFC0000000000)  # bits 42..63: no such cells
    env = L.Env(G.C4, 6, 7, n)
    env.set_state_bits(torch.from_numpy(junk.view(np.int64)), torch.from_numpy(m.view(np.int32)))
    got = env.get_state()[0].cpu().numpy()
    assert (got == s.board).all()
    env.close()


@pytest.mark.parametrize("name,game,rows,cols", [CASES[1], CASES[4], CASES[9]], ids=["c4", "hex11", "draughts"])
def test_rollout_host_matches_device_path(L, name, game, rows, cols):
    """One call with host buffers: the same outcomes and plies as loading the
    packed state on the device and playing it out, and as the oracle."""
    n = 1000
    s = positions(game, rows, cols, n, 23)
    planes_count = 4 if game == G.DRAUGHTS else 2
    p, m = pack_state_bits(s.board, s.to_move, s.ply, s.passes, s.outcome, planes_count)
    hp = torch.from_numpy(p.view(np.int64)).pin_memory()
    hm = torch.from_numpy(m.view(np.int32)).pin_memory()
    ho = torch.empty(n, dtype=torch.int8).pin_memory()
    hpl = torch.empty(n, dtype=torch.int16).pin_memory()
    env = L.Env(game, rows, cols, n, env_offset=9)
    for _ in range(2):  # the second call reuses the staging
        L.ludax_rollout_host(env.handle, hp, hm, 77, ho, hpl)
        env.sync()
    # part-filled warps (8 or 16 lanes holding envs), one thread per env and persistent: the same results
    for cfg in (L.make_cfg(128, 0, 1, 0, 0, 1, 8), L.make_cfg(64, 2, 1, 1, 0, 1, 16)):
        ho2, hpl2 = torch.zeros_like(ho).pin_memory(), torch.zeros_like(hpl).pin_memory()
        L.ludax_rollout_host(env.handle, hp, hm, 77, ho2, hpl2, cfg)
        env.sync()
        assert torch.equal(ho2, ho) and torch.equal(hpl2, hpl)
    # the same with one buffer each way (ludax_rollout_host_packed)
    pb = p.size * 8
    hin = torch.empty(pb + 4 * n, dtype=torch.uint8).pin_memory()
    hin[:pb] = torch.from_numpy(p.view(np.uint8).reshape(-1))
    hin[pb:] = torch.from_numpy(m.view(np.uint8))
    hout = torch.empty(n + (n & 1) + 2 * n, dtype=torch.uint8).pin_memory()
    ho1, hpl1 = hout[:n].view(torch.int8), hout[n + (n & 1):].view(torch.int16)
    L.ludax_rollout_host_packed(env.handle, hin, hout, 77)
    env.sync()
    assert (ho1.numpy() == ho.numpy()).all() and (hpl1.numpy() == hpl.numpy()).all()
    ref = L.Env(game, rows, cols, n, env_offset=9)
    ref.set_state_bits(torch.from_numpy(p.view(np.int64)), torch.from_numpy(m.view(np.int32)))
    o, pl = ref.rollout(77, from_start=False)
    torch.cuda.synchronize()
    assert (ho.numpy() == o.cpu().numpy()).all() and (hpl.numpy() == pl.cpu().numpy()).all()
    t = s.copy()
    G.rollout_from(t, seed=77, env_offset=9)
    assert (ho.numpy() == t.outcome).all() and (hpl.numpy() == t.ply).all()
    for e in (env, ref):
        e.close()


@pytest.mark.parametrize("rows,cols,line,flags", [(9, 12, 5, 0), (8, 9, 5, 3), (10, 11, 4, 2)])
def test_packed_view_line_games(L, rows, cols, line, flags):
    """The parametric line game (run-time board shape, up to 110 cells here: two
    words per plane) through both views."""
    n = 257
    gid = 7 | (line << 8) | (flags << 12)
    s = positions(gid, rows, cols, n, 29)
    view = (s.board, s.to_move, s.ply, s.passes, s.outcome)
    want_p, want_m = pack_state_bits(*view, 2)
    a = L.Env("line", rows, cols, n, env_offset=2, line=line, flags=flags)
    a.set_state(*(torch.from_numpy(x) for x in view))
    p, m = a.get_state_bits()
    torch.cuda.synchronize()
    assert (p.cpu().numpy().view(np.uint64) == want_p).all() and (m.cpu().numpy().view(np.uint32) == want_m).all()
    b = L.Env("line", rows, cols, n, env_offset=2, line=line, flags=flags)
    b.set_state_bits(torch.from_numpy(want_p.view(np.int64)), torch.from_numpy(want_m.view(np.int32)))
    for g_, w_ in zip((t.cpu().numpy() for t in b.get_state()), view):
        assert (g_ == w_).all()
    oa, _ = a.rollout(5, from_start=False)
    ob, _ = b.rollout(5, from_start=False)
    assert (oa.cpu().numpy() == ob.cpu().numpy()).all()
    for e in (a, b):
        e.close()
