"""World-size-2 run of the sharding and aggregation used by bench.py under
torchrun, on CPU with the gloo backend (the ranks play their env ranges
through the oracle; no GPU)."""
import os
import socket

import numpy as np
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank_main(rank, world, port, n_per_rank, q):
    import torch.distributed as dist

    from oracle import games as G
    from paper_2506_22609_b300 import dist as D

    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    r, w, lr = D.world_info()
    off = D.shard_offset(r, n_per_rank)
    out, plies, _ = G.rollout_start(G.C4, 6, 7, n_per_rank, seed=1, env_offset=off)
    # each rank reports a different time; the job time is the max, the work the sum
    t, u = D.aggregate(10.0 + rank, int(plies.astype(np.int64).sum()))
    q.put((r, w, lr, off, out.tolist(), plies.tolist(), t, u))
    dist.barrier()
    dist.destroy_process_group()


def test_two_rank_shards_cover_the_global_batch():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    world, n = 2, 500
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, world, port, n, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in range(world))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    from oracle import games as G

    out_all, plies_all, _ = G.rollout_start(G.C4, 6, 7, world * n, seed=1)
    got_out = np.concatenate([np.array(x[4]) for x in res])
    got_plies = np.concatenate([np.array(x[5]) for x in res])
    assert (got_out == out_all).all() and (got_plies == plies_all).all()
    for r, w, lr, off, *_rest in res:
        assert w == world and lr == r and off == r * n
    t = {x[6] for x in res}
    u = {x[7] for x in res}
    assert t == {11.0} and u == {float(plies_all.astype(np.int64).sum())}


def test_aggregate_is_identity_without_a_process_group():
    from paper_2506_22609_b300 import dist as D

    assert D.aggregate(3.5, 7) == (3.5, 7.0)
    assert D.shard_offset(3, 100) == 300
