"""Compiled game descriptions on the GPU: text -> descriptor -> env and
mixed-batch kernels, compared with the oracle element by element."""
import numpy as np
import pytest
import torch

from oracle import games as G
from paper_2506_22609_b300 import dsl

pytestmark = pytest.mark.gpu

LIB = dsl.library()


def oracle_gid(spec):
    return spec.game if spec.game != dsl.GAME_LINE else 7 | (spec.line << 8) | (spec.flags << 12)


@pytest.mark.parametrize("name", sorted(LIB))
@pytest.mark.parametrize("specialize", [True, False])
def test_compiled_env_matches_oracle(cuda_device, name, specialize):
    spec = dsl.compile_game(LIB[name], specialize=specialize)
    n, seed = (1000 if spec.game == dsl.GAME_PENTE else 4000), 31
    env = dsl.make_env(spec, n, env_offset=3)
    out, plies = env.rollout(seed)
    torch.cuda.synchronize()
    o, p, _ = G.rollout_start(oracle_gid(spec), spec.rows, spec.cols, n, seed, env_offset=3)
    assert (out.cpu().numpy() == o).all() and (plies.cpu().numpy() == p).all()


def test_compiled_library_mixed_batch_matches_oracle(cuda_device):
    from paper_2506_22609_b300 import ludax as L

    descs = [dsl.descriptor(t) for t in LIB.values()] + [dsl.descriptor(t, specialize=False) for t in LIB.values()]
    rng = np.random.default_rng(5)
    n, seed = 30000, 77
    d = np.array(descs, np.int32)[rng.integers(0, len(descs), n)]
    o, p = G.rollout_mixed(d, seed, env_offset=11)
    dd = torch.from_numpy(d).cuda()
    out = torch.empty(n, dtype=torch.int8, device="cuda")
    plies = torch.empty(n, dtype=torch.int16, device="cuda")
    plan = L.ludax_mixed_plan_create(dd, env_offset=11)
    try:
        L.ludax_mixed_plan_launch(plan, seed, out, plies)
        torch.cuda.synchronize()
    finally:
        L.ludax_mixed_plan_destroy(plan)
    assert (out.cpu().numpy() == o).all() and (plies.cpu().numpy() == p).all()


def test_gavel_library_launch_sampled(cuda_device):
    """The GAVEL-like evaluation in the configuration bench.py times: the 13
    library games, each with 100 matches between equal 100-iteration agents,
    50 with the 100-iteration agent moving first against a 50-iteration one
    and 50 the other way round, all 2,600 in one ludax_mcts_play_mixed
    launch; one match per game (the pairings taken in turn) against the
    oracle's match with the same global index."""
    from paper_2506_22609_b300 import ludax as L

    desc, iters, spans = [], [], []
    for name in sorted(LIB):
        spec = dsl.compile_game(LIB[name])
        for n, i1, i2 in ((100, 100, 100), (50, 100, 50), (50, 50, 100)):
            spans.append((name, spec, len(desc), n, i1, i2))
            desc += [spec.desc] * n
            iters += [(i1, i2)] * n
    n, seed = len(desc), 0
    assert n == 2600
    out = torch.empty(n, dtype=torch.int8, device="cuda")
    plies, agency, cov = (torch.empty(n, dtype=torch.int16, device="cuda") for _ in range(3))
    L.ludax_mcts_play_mixed(np.array(desc, np.int32), np.array(iters, np.int32), 0, seed, 2 ** 0.5, out, plies,
                            agency, cov)
    torch.cuda.synchronize()
    got = [t.cpu().numpy() for t in (out, plies, agency, cov)]
    rng = np.random.default_rng(17)
    for g in range(len(LIB)):
        name, spec, first, k, i1, i2 = spans[3 * g + g % 3]
        e = first + int(rng.integers(0, k))
        want = G.mcts_play(oracle_gid(spec), spec.rows, spec.cols, 1, seed, i1, i2, env_offset=e)
        for g_arr, w_arr in zip(got, want):
            assert g_arr[e] == w_arr[0], (name, e)


def test_compiled_library_full_batch_sampled(cuda_device):
    """The compiled-library mix in the configuration bench.py times: 2^20 envs,
    env e playing library game e mod 13, through the autotuned, graph-captured
    mixed plan; sampled envs against the oracle, each with its own index."""
    from paper_2506_22609_b300 import ludax as L
    from paper_2506_22609_b300 import workloads as W

    descs = [dsl.descriptor(t) for t in LIB.values()]
    n, seed = 1 << 20, 3
    d_host = np.array(descs, np.int32)[np.arange(n) % len(descs)]
    d = torch.from_numpy(d_host).cuda()
    cfg, _, _ = L.ludax_autotune(d, seed, reps=1)
    plan = L.ludax_mixed_plan_create(d, 0, cfg)
    out = torch.empty(n, dtype=torch.int8, device="cuda")
    plies = torch.empty(n, dtype=torch.int16, device="cuda")
    try:
        L.ludax_mixed_plan_launch(plan, seed, out, plies)
        torch.cuda.synchronize()
    finally:
        L.ludax_mixed_plan_destroy(plan)
    out, plies = out.cpu().numpy(), plies.cpu().numpy()
    for e in W.sample_envs(n, 650, 23):
        o, p = G.rollout_mixed(d_host[e:e + 1], seed, env_offset=int(e))
        assert o[0] == out[e] and p[0] == plies[e], (int(e), int(d_host[e]))
