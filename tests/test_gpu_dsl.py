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
