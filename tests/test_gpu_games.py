"""GPU parity: the CUDA path (through the C-ABI) against the CPU oracle,
bit-exact on boards, ply counts, outcomes, rewards and legal masks.

Sizes span several 256-thread tiles plus a ragged tail; the benchmark sizes
are checked on sampled envs, which the oracle replays one by one from the
same (seed, global env index).
"""
import numpy as np
import pytest
import torch

from oracle import games as G
from paper_2506_22609_b300 import workloads as W

pytestmark = pytest.mark.gpu

GAMES = [("ttt", G.TTT, 3, 3), ("c4", G.C4, 6, 7), ("othello", G.OTHELLO, 8, 8)] + [
    (f"hex{n}", G.HEX, n, n) for n in (2, 3, 5, 7, 9, 11)] + [
    ("gomoku", G.GOMOKU, 15, 15), ("pente", G.PENTE, 19, 19), ("yavalath", G.YAVALATH, 9, 9)]
BIG = (G.GOMOKU, G.PENTE)


def cells_of(game, rows, cols):
    return G.num_cells(game, rows, cols)
GAME_IDS = [g[0] for g in GAMES]


@pytest.fixture(scope="module")
def L(cuda_device):
    from paper_2506_22609_b300 import build

    build.build()
    from paper_2506_22609_b300 import ludax

    ludax.lib()
    return ludax


def np_(t):
    return t.detach().cpu().numpy()


def gpu_state(env):
    b, tm, ply, ps, oc = env.get_state()
    torch.cuda.synchronize()
    return np_(b), np_(tm), np_(ply), np_(ps), np_(oc)


def assert_states_equal(env, s):
    b, tm, ply, ps, oc = gpu_state(env)
    assert (b == s.board).all()
    assert (tm == s.to_move).all()
    assert (ply == s.ply).all()
    assert (ps == s.passes).all()
    assert (oc == s.outcome).all()


# ---------------------------------------------------------------- rollouts --
@pytest.mark.parametrize("name,game,rows,cols", GAMES, ids=GAME_IDS)
def test_rollout_from_start_matches_oracle(L, name, game, rows, cols):
    n, seed, off = (700 if game in BIG else 2600), 7, 12345
    env = L.Env(game, rows, cols, n, env_offset=off)
    out, plies = env.rollout(seed, from_start=True, write_back=True)
    o_out, o_plies, o_boards = G.rollout_start(game, rows, cols, n, seed, env_offset=off, want_boards=True)
    assert (np_(out) == o_out).all()
    assert (np_(plies) == o_plies).all()
    b, tm, ply, ps, oc = gpu_state(env)
    assert (b == o_boards).all()
    assert (oc == o_out).all() and (ply == o_plies).all()
    assert env.counters() == (0, 0)
    assert set(np.unique(o_out)) <= {0, 1, 2}


@pytest.mark.parametrize("cfg", [(256, 0, 1, 0, 0), (128, 2, 1, 0, 0), (64, 1, 2, 1, 0), (512, 4, 2, 0, 0),
                                 (96, 3, 1, 1, 0), (256, 0, 1, 0, 4), (128, 2, 1, 1, 8), (448, 1, 1, 0, 16),
                                 (64, 1, 1, 0, 1)],
                         ids=lambda c: "b{}_bps{}_ept{}_tab{}_cmp{}".format(*c))
@pytest.mark.parametrize("name,game,rows,cols", [GAMES[1], GAMES[2], GAMES[7], GAMES[8], GAMES[10], GAMES[11]],
                         ids=["c4", "othello", "hex9", "hex11", "pente", "yavalath"])
def test_launch_shape_does_not_change_results(L, name, game, rows, cols, cfg):
    # persistent grids smaller than the batch exercise the refill path
    n, seed = (6000 if game in BIG else 20000), 3
    env = L.Env(game, rows, cols, n)
    out, plies = env.rollout(seed, cfg=L.make_cfg(*cfg))
    ref_out, ref_plies = env.rollout(seed)
    torch.cuda.synchronize()
    assert torch.equal(out, ref_out) and torch.equal(plies, ref_plies)
    s = W.sample_envs(n, 400, 1)
    for e in s[:50]:
        o, p, _ = G.rollout_start(game, rows, cols, 1, seed, env_offset=int(e))
        assert o[0] == np_(out)[e] and p[0] == np_(plies)[e]


# part-filled warps: only the first 8 or 16 lanes of each warp hold envs, one
# thread per env or persistent (refilling), one or two envs per thread
@pytest.mark.parametrize("cfg", [(256, 0, 1, 0, 0, 1, 8), (128, 0, 2, 1, 0, 1, 16), (64, 2, 1, 1, 0, 1, 8),
                                 (512, 1, 2, 0, 0, 1, 16), (32, 0, 1, 0, 0, 1, 16)],
                         ids=lambda c: "b{}_bps{}_ept{}_tab{}_lanes{}".format(c[0], c[1], c[2], c[3], c[6]))
@pytest.mark.parametrize("name,game,rows,cols", [GAMES[0], GAMES[1], GAMES[2], GAMES[8], GAMES[11]],
                         ids=["ttt", "c4", "othello", "hex11", "yavalath"])
def test_part_filled_warps_match_oracle(L, name, game, rows, cols, cfg):
    n, seed, off = (700 if game in BIG else 3001), 9, 321
    env = L.Env(game, rows, cols, n, env_offset=off)
    out, plies = env.rollout(seed, from_start=True, write_back=True, cfg=L.make_cfg(*cfg))
    o_out, o_plies, o_boards = G.rollout_start(game, rows, cols, n, seed, env_offset=off, want_boards=True)
    assert (np_(out) == o_out).all() and (np_(plies) == o_plies).all()
    b, tm, ply, ps, oc = gpu_state(env)
    assert (b == o_boards).all() and (oc == o_out).all()
    assert env.counters() == (0, 0)


def test_part_filled_warps_argument_checks(L):
    env = L.Env("hex", 7, 7, 64)
    for bad in [(64, 0, 1, 0, 0, 1, 4), (64, 0, 1, 0, 0, 1, 24), (64, 0, 1, 0, 4, 1, 8), (64, 0, 1, 0, 0, 2, 8)]:
        with pytest.raises(L.LudaxError) as ei:  # 8, 16 or 32 lanes; no compaction, one lane per env
            env.rollout(1, cfg=L.make_cfg(*bad))
        assert ei.value.status == -1
    with pytest.raises(L.LudaxError):  # the value playouts run full warps
        env.rollout_value(1, 4, cfg=L.make_cfg(64, 0, 1, 0, 0, 1, 8))
    env.close()


@pytest.mark.parametrize("n", [1, 31, 33, 257])
def test_ragged_and_tiny_batches(L, n):
    for name, game, rows, cols in (GAMES[0], GAMES[1], GAMES[2], GAMES[8], GAMES[9], GAMES[11]):
        env = L.Env(game, rows, cols, n)
        o, p, _ = G.rollout_start(game, rows, cols, n, 11)
        for cfg in [(64, 1, 2, 0, 0), (64, 1, 1, 0, 4), (32, 1, 1, 1, 2), (64, 0, 1, 0, 0, 1, 8)]:
            out, plies = env.rollout(11, cfg=L.make_cfg(*cfg))
            assert (np_(out) == o).all() and (np_(plies) == p).all()


# ------------------------------------------------- benchmark-size configs --
@pytest.mark.parametrize("cfg", [W.TTT_1K, W.C4_64K, W.OTHELLO_256K, W.HEX11_64K, W.GOMOKU_64K, W.PENTE_64K,
                                 W.YAVALATH_64K], ids=lambda c: c.name)
def test_benchmark_configs_sampled(L, cfg):
    env = L.Env(cfg.game, cfg.rows, cfg.cols, cfg.num_envs)
    out, plies = env.rollout(cfg.seed, cfg=L.make_cfg(*W.bench_cfg(cfg)))
    out, plies = np_(out), np_(plies)
    if cfg.num_envs <= 65536 and cfg.game in (G.TTT, G.C4):
        o, p, _ = G.rollout_start(cfg.game, cfg.rows, cfg.cols, cfg.num_envs, cfg.seed)
        assert (out == o).all() and (plies == p).all()
    else:
        for e in W.sample_envs(cfg.num_envs, 300 if cfg.game in BIG else 1500, 5):
            o, p, _ = G.rollout_start(cfg.game, cfg.rows, cfg.cols, 1, cfg.seed, env_offset=int(e))
            assert o[0] == out[e] and p[0] == plies[e], e
    assert set(np.unique(out)) <= {0, 1, 2}
    # properties that hold at any size: length bounds and the winner moved last
    lo, hi = {G.TTT: (5, 9), G.C4: (7, 42), G.OTHELLO: (11, 128), G.HEX: (2 * cfg.rows - 1, cfg.rows ** 2),
              G.GOMOKU: (9, 225), G.PENTE: (9, 2000), G.YAVALATH: (5, 61)}[cfg.game]
    assert plies.min() >= lo and plies.max() <= hi
    if cfg.game in (G.TTT, G.C4, G.HEX, G.GOMOKU, G.PENTE):
        won = out != 0
        assert ((plies[won] % 2 == 1) == (out[won] == 1)).all()
    if cfg.game == G.HEX:
        assert (out != 0).all()


@pytest.mark.parametrize("cfg", [W.CONNECT5_9X12_64K, W.WOLF_SHEEP_64K, W.DRAUGHTS_64K, W.HASAMI_64K],
                         ids=lambda c: c.name)
def test_benchmark_extra_configs_sampled(L, cfg):
    """The other playout workloads bench.py times, at their size and in their
    launch shape: sampled envs against the oracle, each replayed with its own
    env index (outcome and length, including games ended by the ply cap)."""
    env = L.Env(cfg.game, cfg.rows, cfg.cols, cfg.num_envs, line=cfg.line, flags=cfg.flags)
    out, plies = env.rollout(cfg.seed, cfg=L.make_cfg(*W.bench_cfg(cfg)))
    out, plies = np_(out), np_(plies)
    gid = line_gid(cfg.line, cfg.flags) if cfg.line else cfg.game
    for e in W.sample_envs(cfg.num_envs, 400, 9):
        o, p, _ = G.rollout_start(gid, cfg.rows, cfg.cols, 1, cfg.seed, env_offset=int(e))
        assert o[0] == out[e] and p[0] == plies[e], e
    assert plies.min() >= 1 and plies.max() <= G.ply_cap(gid, cfg.rows, cfg.cols)
    env.close()


# ------------------------------------------------------ step-per-launch --
@pytest.mark.parametrize("name,game,rows,cols", GAMES, ids=GAME_IDS)
def test_random_step_reproduces_rollout(L, name, game, rows, cols):
    n, seed = (300 if game in BIG else 1500), 21
    env = L.Env(game, rows, cols, n, env_offset=99)
    ref = L.Env(game, rows, cols, n, env_offset=99)
    r_out, r_plies = ref.rollout(seed, write_back=True)
    done = torch.zeros(n, dtype=torch.bool, device="cuda")
    cap = G.ply_cap(game, rows, cols)
    final_rew = torch.zeros(n, 2, device="cuda")
    for _ in range(cap + 2):
        rew, term = env.random_step(seed)
        newly = term.bool() & ~done
        final_rew[newly] = rew[newly]
        assert (rew[~newly] == 0).all()
        done |= term.bool()
        if bool(done.all()):
            break
    assert bool(done.all())
    b1 = gpu_state(env)
    b2 = gpu_state(ref)
    for x, y in zip(b1, b2):
        assert (x == y).all()
    want = np.zeros((n, 2), np.float32)
    ro = np_(r_out)
    want[ro == 1] = (1, -1)
    want[ro == 2] = (-1, 1)
    assert (np_(final_rew) == want).all()


def test_step_mode_full_size_sampled(L):
    """The step-per-launch benchmark configuration: 16,777,216 Connect Four
    envs, reset, then five ludax_random_step launches over the whole batch;
    sampled envs against the oracle's playout stopped after five plies, and
    at any size: no game ends before ply 7, so every reward and flag is 0."""
    n, seed, plies = 1 << 24, 1, 5
    env = L.Env(G.C4, 6, 7, n)
    for _ in range(plies):
        rew, term = env.random_step(seed)
    assert bool((rew == 0).all()) and bool((term == 0).all())
    b, tm, ply, ps, oc = env.get_state()
    idx = torch.from_numpy(W.sample_envs(n, 2000, 7)).cuda()
    b, tm, ply, ps, oc = (np_(t[idx]) for t in (b, tm, ply, ps, oc))
    assert (ply == plies).all() and (oc == -1).all()
    for i, e in enumerate(np_(idx)):
        s = G.reset(G.C4, 6, 7, 1)
        G.rollout_from(s, seed, env_offset=int(e), stop_ply=np.array([plies], np.int16))
        assert (s.board[0] == b[i]).all() and s.to_move[0] == tm[i] and s.ply[0] == ply[i], int(e)
    env.close()


def _canon_legal(mask_words, A, cells):
    bits = np.zeros((mask_words.shape[0], A), np.uint8)
    w = mask_words.view(np.uint64)
    for c in range(cells):
        bits[:, c] = (w[:, c // 64] >> np.uint64(c % 64)) & np.uint64(1)
    return bits


@pytest.mark.parametrize("name,game,rows,cols", GAMES, ids=GAME_IDS)
def test_step_api_matches_oracle(L, name, game, rows, cols):
    # Oracle-chosen trajectories, 10% of steps with an arbitrary (often
    # illegal) action: legal masks, rewards, terminated flags and full state
    # must agree after every step.
    n = 128 if game in BIG else 700
    rng = np.random.default_rng(game * 100 + rows)
    env = L.Env(game, rows, cols, n)
    s = G.reset(game, rows, cols, n)
    A, cells = G.num_actions(game, rows, cols), cells_of(game, rows, cols)
    assert env.num_actions == A
    n_illegal = 0
    for _ in range(cells * 2 + 4):
        legal = G.legal(s)
        m, p = env.legal_mask()
        torch.cuda.synchronize()
        got = _canon_legal(np_(m), A, cells)
        if game == G.OTHELLO:
            got[:, cells] = np_(p)
        else:
            assert not np_(p).any()
        assert (got == legal).all()
        acts = np.zeros(n, np.int32)
        for e in range(n):
            cand = np.flatnonzero(legal[e])
            if cand.size == 0 or rng.random() < 0.1:
                acts[e] = rng.integers(-2, A + 2)
            else:
                acts[e] = rng.choice(cand)
        o_rew, o_term, o_err = G.step(s, acts)
        n_illegal += int(o_err.sum())
        rew, term = env.step(torch.from_numpy(acts).cuda())
        torch.cuda.synchronize()
        assert (np_(rew) == o_rew).all()
        assert (np_(term) == o_term).all()
        assert_states_equal(env, s)
        if o_term.all():
            break
    assert s.outcome.min() >= 0
    assert env.counters()[0] == n_illegal and n_illegal > 0


def test_reset_mask_and_finished_env_noop(L):
    env = L.Env("c4", 6, 7, 64)
    env.rollout(5, write_back=True)
    mask = torch.zeros(64, dtype=torch.uint8, device="cuda")
    mask[::2] = 1
    env.reset(mask)
    b, tm, ply, ps, oc = gpu_state(env)
    assert (b[::2] == 0).all() and (ply[::2] == 0).all() and (oc[::2] == -1).all()
    assert (oc[1::2] >= 0).all()
    before = gpu_state(env)
    rew, term = env.step(torch.zeros(64, dtype=torch.int32, device="cuda") + 38)
    after = gpu_state(env)
    for x, y in zip(before, after):
        assert (x[1::2] == y[1::2]).all()
    assert (np_(rew)[1::2] == 0).all() and np_(term)[1::2].all()


# --------------------------------------------------- positions and values --
@pytest.mark.parametrize("name,game,rows,cols", GAMES, ids=GAME_IDS)
def test_set_state_rollout_from_positions(L, name, game, rows, cols):
    n = 300 if game in BIG else 1200
    rng = np.random.default_rng(rows + 17 * game)
    s = G.reset(game, rows, cols, n)
    stop = rng.integers(0, cells_of(game, rows, cols), n).astype(np.int16)
    G.rollout_from(s, seed=5, stop_ply=stop)
    env = L.Env(game, rows, cols, n, env_offset=7)
    env.set_state(*(torch.from_numpy(x) for x in (s.board, s.to_move, s.ply, s.passes, s.outcome)))
    assert_states_equal(env, s)
    # partial playouts to a stop ply, then to the end, from the stored state
    s2 = s.copy()
    stop2 = (s.ply + rng.integers(0, 6, n)).astype(np.int16)
    G.rollout_from(s2, seed=9, env_offset=7, stop_ply=stop2)
    out, plies = env.rollout(9, from_start=False, write_back=True, stop_ply=torch.from_numpy(stop2).cuda())
    assert_states_equal(env, s2)
    assert (np_(out) == s2.outcome).all() and (np_(plies) == s2.ply).all()
    G.rollout_from(s2, seed=10, env_offset=7)
    out, plies = env.rollout(10, from_start=False, write_back=True)
    assert_states_equal(env, s2)


@pytest.mark.parametrize("name,game,rows,cols", [GAMES[1], GAMES[2], GAMES[8]], ids=["c4", "othello", "hex11"])
def test_rollout_value_matches_oracle(L, name, game, rows, cols):
    n, R, seed = 300, 16, 1000
    s = G.reset(game, rows, cols, n)
    G.rollout_from(s, seed=3, stop_ply=np.full(n, 10, np.int16))
    env = L.Env(game, rows, cols, n, env_offset=50)
    env.set_state(*(torch.from_numpy(x) for x in (s.board, s.to_move, s.ply, s.passes, s.outcome)))
    v = np_(env.rollout_value(seed, R))
    acc = np.zeros(n)
    for j in range(R):
        t = s.copy()
        G.rollout_from(t, seed=seed + j, env_offset=50)
        acc += np.where(t.outcome == 1, 1.0, np.where(t.outcome == 2, 0.0, 0.5))
    assert (v == (acc / R).astype(np.float32)).all()
    assert_states_equal(env, s)  # the stored state is untouched


# ------------------------------------------------------------ mixed batch --
@pytest.mark.parametrize("layout", ["block", "interleave", "random"])
def test_mixed_batch_matches_oracle(L, layout):
    n, seed, off = 6000, 3, 777
    d = W.random_descriptors(n, 4) if layout == "random" else W.mixed_descriptors(n, layout)
    o_out, o_plies = G.rollout_mixed(d, seed, env_offset=off)
    dd = torch.from_numpy(d).cuda()
    out = torch.empty(n, dtype=torch.int8, device="cuda")
    plies = torch.empty(n, dtype=torch.int16, device="cuda")
    L.ludax_rollout_mixed(dd, off, seed, out, plies)
    torch.cuda.synchronize()
    assert (np_(out) == o_out).all() and (np_(plies) == o_plies).all()
    # persistent shapes, one thread per env, two interleaved envs per thread, part-filled warps
    for cfg in [(128, 2, 1, 1, 0), (64, 1, 1, 0, 0), (512, 0, 1, 1, 0), (256, 4, 1, 0, 0), (32, 1, 1, 1, 0),
                (128, 0, 2, 1, 0), (64, 0, 1, 0, 0, 1, 16), (256, 0, 2, 1, 0, 1, 8), (96, 0, 2, 0, 0, 1, 16)]:
        plan = L.ludax_mixed_plan_create(dd, off, L.make_cfg(*cfg))
        for s2 in (seed, seed + 1):
            out2 = torch.full((n,), 99, dtype=torch.int8, device="cuda")
            plies2 = torch.zeros(n, dtype=torch.int16, device="cuda")
            L.ludax_mixed_plan_launch(plan, s2, out2, plies2)
            torch.cuda.synchronize()
            if s2 == seed:
                assert torch.equal(out2, out) and torch.equal(plies2, plies)
            else:
                o2, p2 = G.rollout_mixed(d, s2, env_offset=off)
                assert (np_(out2) == o2).all() and (np_(plies2) == p2).all()
        L.ludax_mixed_plan_destroy(plan)


def test_mixed_full_config_sampled(L):
    d = W.mixed_descriptors(W.MIXED_ENVS, "block")
    dd = torch.from_numpy(d).cuda()
    plan = L.ludax_mixed_plan_create(dd, 0, L.make_cfg(*W.mixed_bench_cfg()))
    out = torch.empty(W.MIXED_ENVS, dtype=torch.int8, device="cuda")
    plies = torch.empty(W.MIXED_ENVS, dtype=torch.int16, device="cuda")
    L.ludax_mixed_plan_launch(plan, W.MIXED_SEED, out, plies)
    torch.cuda.synchronize()
    out, plies = np_(out), np_(plies)
    for e in W.sample_envs(W.MIXED_ENVS, 1200, 9):
        o, p = G.rollout_mixed(d[e:e + 1], W.MIXED_SEED, env_offset=int(e))
        assert o[0] == out[e] and p[0] == plies[e], e
    assert set(np.unique(out)) <= {0, 1, 2}
    L.ludax_mixed_plan_destroy(plan)


@pytest.mark.parametrize("cfg", [(128, 0, 1, 1, 0), (128, 2, 1, 1, 0), (256, 0, 2, 1, 0, 1, 16)])
def test_mixed_host_buffers_match_oracle(L, cfg):
    # the plan's host-buffer launch: descriptors uploaded, queue rebuilt on the
    # device, results copied back; any batch of the plan's size, including ones
    # the plan was not built from, and invalid descriptors reported by sync
    n, off = 3001, 55
    d0 = W.mixed_descriptors(n, "block")
    plan = L.ludax_mixed_plan_create(torch.from_numpy(d0).cuda(), off, L.make_cfg(*cfg))
    h_out = torch.empty(n, dtype=torch.int8).pin_memory()
    h_plies = torch.empty(n, dtype=torch.int16).pin_memory()
    for k, (d, seed) in enumerate(((W.random_descriptors(n, 5), 3), (W.mixed_descriptors(n, "interleave"), 4),
                                   (d0, 5))):
        h_desc = torch.from_numpy(d).pin_memory()
        L.ludax_mixed_plan_launch_host(plan, seed, h_desc, h_out, h_plies)
        L.ludax_mixed_plan_sync(plan)
        o, p = G.rollout_mixed(d, seed, env_offset=off)
        assert (h_out.numpy() == o).all() and (h_plies.numpy() == p).all(), k
    # the captured graph keeps its own queue
    out = torch.empty(n, dtype=torch.int8, device="cuda")
    plies = torch.empty(n, dtype=torch.int16, device="cuda")
    L.ludax_mixed_plan_launch(plan, 5, out, plies)
    torch.cuda.synchronize()
    assert (np_(out) == h_out.numpy()).all() and (np_(plies) == h_plies.numpy()).all()
    bad = W.mixed_descriptors(n, "interleave")
    bad[2500], bad[1999] = W.desc(3, 12, 12), W.desc(11, 3, 3)
    L.ludax_mixed_plan_launch_host(plan, 6, torch.from_numpy(bad).pin_memory(), h_out, h_plies)
    with pytest.raises(L.LudaxError) as ei:
        L.ludax_mixed_plan_sync(plan)
    assert ei.value.status == -2 and ei.value.bad_index == 1999
    good = np.ones(n, bool)
    good[[1999, 2500]] = False
    # the valid envs are played as usual (their draws are keyed by their own index)
    idx = np.nonzero(good)[0]
    for j in W.sample_envs(len(idx), 200, 3):
        e = int(idx[j])
        oe, pe = G.rollout_mixed(bad[e:e + 1], 6, env_offset=off + e)
        assert h_out.numpy()[e] == oe[0] and h_plies.numpy()[e] == pe[0]
    assert h_out.numpy()[1999] == -1 and h_plies.numpy()[2500] == 0
    L.ludax_mixed_plan_destroy(plan)


def test_mixed_rejects_bad_descriptors(L):
    d = W.mixed_descriptors(100, "block")
    d[37] = W.desc(3, 12, 12)
    with pytest.raises(L.LudaxError) as ei:
        L.ludax_mixed_plan_create(torch.from_numpy(d).cuda())
    assert ei.value.status == -3 and ei.value.bad_index == 37
    d[37] = W.desc(11, 3, 3)                      # no game has id 11
    with pytest.raises(L.LudaxError) as ei:
        L.ludax_mixed_plan_create(torch.from_numpy(d).cuda())
    assert ei.value.status == -2
    d[37] = W.desc(7, 6, 7)                       # line game without a line length
    with pytest.raises(L.LudaxError) as ei:
        L.ludax_mixed_plan_create(torch.from_numpy(d).cuda())
    assert ei.value.status == -3


def test_sync_deadline_returns_timeout_status(L):
    env = L.Env("othello", 8, 8, 262144)
    saw_timeout = False
    for _ in range(3):
        env.rollout(1)
        st = L.lib().ludax_sync(env.handle, 0)
        assert st in (0, -5)
        saw_timeout |= st == -5
        env.sync(60000)
    assert saw_timeout


# ------------------------------------------------- parametric line game --
LINE_CASES = [(3, 3, 3, 0), (6, 7, 4, 2), (4, 4, 3, 4), (7, 7, 4, 1), (9, 12, 5, 0), (8, 9, 5, 3), (1, 8, 3, 0)]


def line_gid(line, flags):
    """The oracle's id for a parametric line game."""
    return 7 | (line << 8) | (flags << 12)


@pytest.mark.parametrize("rows,cols,line,flags", LINE_CASES, ids=lambda *a: None)
def test_line_game_matches_oracle(L, rows, cols, line, flags):
    n, seed, off = 2000, 13, 5
    env = L.Env("line", rows, cols, n, env_offset=off, line=line, flags=flags)
    assert env.num_actions == rows * cols
    out, plies = env.rollout(seed, write_back=True)
    o, p, b = G.rollout_start(line_gid(line, flags), rows, cols, n, seed, env_offset=off, want_boards=True)
    assert (np_(out) == o).all() and (np_(plies) == p).all()
    assert (gpu_state(env)[0] == b).all()
    # oracle-driven trajectories through the step API, legal masks each ply
    m = 200
    env2 = L.Env("line", rows, cols, m, line=line, flags=flags)
    s = G.reset(line_gid(line, flags), rows, cols, m)
    rng = np.random.default_rng(rows * 31 + cols)
    for _ in range(rows * cols + 1):
        legal = G.legal(s)
        mk, _pass = env2.legal_mask()
        torch.cuda.synchronize()
        assert (_canon_legal(np_(mk), rows * cols, rows * cols) == legal).all()
        acts = np.array([rng.choice(np.flatnonzero(lg)) if lg.any() else 0 for lg in legal], np.int32)
        o_rew, o_term, _ = G.step(s, acts)
        rew, term = env2.step(torch.from_numpy(acts).cuda())
        torch.cuda.synchronize()
        assert (np_(rew) == o_rew).all() and (np_(term) == o_term).all()
        assert_states_equal(env2, s)
        if o_term.all():
            break


def test_mixed_batch_with_line_games(L):
    n, seed = 4000, 21
    rng = np.random.default_rng(3)
    pool = [L.LUDAX_DESC_LINE(r, c, ln, fl) for r, c, ln, fl in LINE_CASES] + [
        W.desc(0, 3, 3), W.desc(1, 6, 7), W.desc(3, 7, 7), W.desc(6, 9, 9)]
    d = np.array(pool, np.int32)[rng.integers(0, len(pool), n)]
    o, p = G.rollout_mixed(d, seed)
    dd = torch.from_numpy(d).cuda()
    out = torch.empty(n, dtype=torch.int8, device="cuda")
    plies = torch.empty(n, dtype=torch.int16, device="cuda")
    plan = L.ludax_mixed_plan_create(dd)
    L.ludax_mixed_plan_launch(plan, seed, out, plies)
    torch.cuda.synchronize()
    assert (np_(out) == o).all() and (np_(plies) == p).all()
    L.ludax_mixed_plan_destroy(plan)
    bad = d.copy()
    bad[7] = L.LUDAX_DESC_LINE(12, 12, 5, 0)       # 12 x 13 > 128 padded cells
    with pytest.raises(L.LudaxError) as ei:
        L.ludax_mixed_plan_create(torch.from_numpy(bad).cuda())
    assert ei.value.status == -3 and ei.value.bad_index == 7
