"""The allocation-free mixed-batch playout (ludax_rollout_mixed_noalloc).

It exists for callers that cannot allocate device memory -- a plugin inside a
host framework whose memory pool owns the device's memory, or a serving loop
that must not let cudaFree synchronise the device.  Its scratch is a static
device array shared by every call, so this test calls it twice in a row (the
second call must not see the first call's queue or counters) and checks each
result against the allocating entry point ludax_rollout_mixed, exactly:
outcomes and game lengths are integers.  It also checks that the device's
free memory does not move across calls once the kernels are loaded.  This
file is collected last on purpose.
"""
import pytest
import torch

from paper_2506_22609_b300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def L(cuda_device):
    from paper_2506_22609_b300 import build

    build.build()
    from paper_2506_22609_b300 import ludax

    ludax.lib()
    return ludax


def run_both(L, d, off, seed, cfg=None):
    n = d.numel()
    ref_o = torch.empty(n, dtype=torch.int8, device="cuda")
    ref_p = torch.empty(n, dtype=torch.int16, device="cuda")
    L.ludax_rollout_mixed(d, off, seed, ref_o, ref_p, cfg)
    out_o = torch.full((n,), 99, dtype=torch.int8, device="cuda")
    out_p = torch.full((n,), -7, dtype=torch.int16, device="cuda")
    L.ludax_rollout_mixed_noalloc(d, off, seed, out_o, out_p, cfg)
    torch.cuda.synchronize()
    return (ref_o, ref_p), (out_o, out_p)


@pytest.mark.parametrize("layout", ["interleave", "random"])
def test_noalloc_matches_allocating_entry_point_twice(L, layout):
    # two different batches back to back: the second call must rebuild the
    # shared queue and counters from scratch
    d1 = W.mixed_descriptors(5000, "interleave") if layout == "interleave" else W.random_descriptors(5000, 1)
    d2 = W.random_descriptors(3001, 2)
    for d, off, seed in ((d1, 0, 3), (d2, 123, 4)):
        dd = torch.from_numpy(d).cuda()
        (ro, rp), (oo, op) = run_both(L, dd, off, seed)
        assert torch.equal(oo, ro) and torch.equal(op, rp)


def test_noalloc_full_config_and_persistent_shape(L):
    d = torch.from_numpy(W.mixed_descriptors(W.MIXED_ENVS, "block")).cuda()
    for cfg in (L.make_cfg(*W.mixed_bench_cfg()), L.make_cfg(128, 2, 1, 1, 0)):
        (ro, rp), (oo, op) = run_both(L, d, 0, W.MIXED_SEED, cfg)
        assert torch.equal(oo, ro) and torch.equal(op, rp)


def test_noalloc_rejects_oversized_and_bad_batches(L):
    n = (1 << 20) + 1
    d = torch.from_numpy(W.mixed_descriptors(n, "block")).cuda()
    o = torch.empty(n, dtype=torch.int8, device="cuda")
    p = torch.empty(n, dtype=torch.int16, device="cuda")
    with pytest.raises(L.LudaxError) as ei:
        L.ludax_rollout_mixed_noalloc(d, 0, 1, o, p)
    assert ei.value.status == -3
    bad = W.mixed_descriptors(64, "block")
    bad[17] = W.desc(3, 13, 13)
    bad[40] = 9
    with pytest.raises(L.LudaxError) as ei:
        L.ludax_rollout_mixed_noalloc(torch.from_numpy(bad).cuda(), 0, 1, o[:64], p[:64])
    assert ei.value.status == -3 and ei.value.bad_index == 17
    # and the next valid call is unaffected
    good = torch.from_numpy(W.mixed_descriptors(640, "interleave")).cuda()
    (ro, rp), (oo, op) = run_both(L, good, 0, 5)
    assert torch.equal(oo, ro) and torch.equal(op, rp)


def test_noalloc_leaves_device_memory_unchanged(L):
    # after one warm-up call (which loads the kernels it launches), further
    # calls must not change the device's free memory: no allocation, no free
    n = 1 << 20
    d = torch.from_numpy(W.mixed_descriptors(n, "block")).cuda()
    o = torch.empty(n, dtype=torch.int8, device="cuda")
    p = torch.empty(n, dtype=torch.int16, device="cuda")
    cfg = L.make_cfg(*W.mixed_bench_cfg())
    L.ludax_rollout_mixed_noalloc(d, 0, 7, o, p, cfg)
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    for seed in (8, 9, 10):
        L.ludax_rollout_mixed_noalloc(d, 0, seed, o, p, cfg)
        torch.cuda.synchronize()
        assert torch.cuda.mem_get_info()[0] == free0
