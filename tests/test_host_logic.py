"""Host-side logic without a GPU: the CPU baseline's sampling of the mixed
batch, the value net's selection of K and M on validation errors, the
known-answer fixture of the policy's draw (regenerated by its script), and
the value net's checkpoint file format."""
import os
import subprocess
import sys

import numpy as np
import pytest

from conftest import ROOT


def test_cpu_sample_covers_every_game_of_the_mixed_batch():
    sys.path.insert(0, ROOT)
    import bench
    from paper_2506_22609_b300 import workloads as W

    d = W.mixed_descriptors(W.MIXED_ENVS, "block")
    cfg = bench.W_mixed_cfg(W)
    ranges = bench.sample_ranges(cfg, 6000, d)
    assert len(ranges) == len(W.MIXED_GAMES)
    games = {int(d[off]) for off, k in ranges}
    assert games == {W.desc(*g) for g in W.MIXED_GAMES}
    for off, k in ranges:  # each range stays inside one game block
        assert k == 1000 and len(set(d[off:off + k].tolist())) == 1
    assert bench.sample_ranges(W.C4_64K, 5000) == [(0, 5000)]


def test_value_net_selection_takes_the_smallest_count_meeting_the_target():
    sys.path.insert(0, ROOT)
    from paper_2506_22609_b300 import valuenet as V

    rows = [{"K": 1, "mae": 0.09}, {"K": 2, "mae": 0.06}, {"K": 4, "mae": 0.049}, {"K": 8, "mae": 0.04}]
    assert V.first_at(rows, 0.05)["K"] == 4
    assert V.first_at(rows, 0.01)["K"] == 8  # none meets it: the largest count
    assert V.first_at(rows, 0.1)["K"] == 1


def test_draw_fixture_is_what_its_script_writes(tmp_path):
    script = os.path.join(ROOT, "tests", "golden", "make_splitmix64_keys.py")
    fixture = os.path.join(ROOT, "tests", "golden", "splitmix64_keys.txt")
    before = open(fixture).read()
    subprocess.run([sys.executable, script], check=True, capture_output=True)
    assert open(fixture).read() == before
    rows = [l.split() for l in before.splitlines() if l and not l.startswith("#")]
    assert len({(r[0], r[1]) for r in rows}) >= 10 and np.all([len(r) == 7 for r in rows])


def test_value_net_checkpoint_file_round_trip(tmp_path):
    """The checkpoint format on its own (host side): header fields and the
    three arrays come back bit for bit; other files are refused."""
    import numpy as np

    from paper_2506_22609_b300 import valuenet as V

    rng = np.random.default_rng(3)
    n = 1000
    p, m, v = (rng.standard_normal(n).astype(np.float32) for _ in range(3))
    path = str(tmp_path / "net.ckpt")
    V.write_checkpoint(path, 64, 256, 512, 17, p, m, v)
    c = V.read_checkpoint(path)
    assert (c["cells"], c["in_pad"], c["hidden"], c["steps"]) == (64, 256, 512, 17)
    for k, a in (("params", p), ("m", m), ("v", v)):
        assert c[k].dtype == np.float32 and (c[k].view(np.uint32) == a.view(np.uint32)).all()
    data = open(path, "rb").read()
    assert len(data) == 8 + 6 * 8 + 3 * 4 * n
    bad = tmp_path / "bad.ckpt"
    for blob in (b"NOTANET!" + data[8:], data[:-4], data[:8] + (2).to_bytes(8, "little") + data[16:]):
        bad.write_bytes(blob)
        with pytest.raises(ValueError):
            V.read_checkpoint(str(bad))
    with pytest.raises(ValueError):  # moments of another length
        V.write_checkpoint(path, 64, 256, 512, 0, p, m[:-1], v)
