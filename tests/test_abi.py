"""The C-ABI library builds, loads and exports every symbol include/ludax.h
declares; host-side argument validation returns status codes without a GPU.
"""
import ctypes
import os
import re
import subprocess

import pytest

from conftest import ROOT

HEADER = os.path.join(ROOT, "include", "ludax.h")


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"^\s*(?:const\s+)?\w+\s*\*?\s*(ludax_\w+)\s*\(", text, flags=re.M)))


@pytest.fixture(scope="module")
def L():
    from paper_2506_22609_b300 import build, ludax

    build.build()
    return ludax.lib()


def test_header_declares_core_api():
    names = declared_functions()
    for core in ("ludax_env_create", "ludax_env_destroy", "ludax_reset", "ludax_legal_mask", "ludax_step",
                 "ludax_random_step", "ludax_rollout", "ludax_get_state", "ludax_set_state", "ludax_sync",
                 "ludax_status_string", "ludax_mixed_plan_create", "ludax_autotune"):
        assert core in names


def test_every_declared_symbol_is_exported(L):
    from paper_2506_22609_b300 import ludax

    out = subprocess.run(["nm", "-D", "--defined-only", ludax.LIB_PATH], capture_output=True, text=True).stdout
    exported = set(re.findall(r"\bT (ludax_\w+)", out))
    missing = [n for n in declared_functions() if n not in exported]
    assert not missing, missing
    for n in declared_functions():
        getattr(L, n)  # resolvable through ctypes too


def test_build_targets_sm103a_only():
    from paper_2506_22609_b300 import build

    assert build.ARCH == ["-gencode", "arch=compute_103a,code=sm_103a"]


def test_status_strings(L):
    from paper_2506_22609_b300 import ludax

    assert ludax.status_string(0) == "ok"
    for code in range(-7, 0):
        assert ludax.status_string(code) not in ("", "unknown status")
    assert ludax.status_string(-99) == "unknown status"


def test_env_create_rejects_bad_arguments_before_touching_the_device(L):
    from paper_2506_22609_b300 import ludax

    h = ctypes.c_void_p()
    p = ludax.ludax_board_params(6, 7)
    assert L.ludax_env_create(None, 1, ctypes.byref(p), 16, 0, None) == -1
    assert L.ludax_env_create(ctypes.byref(h), 1, None, 16, 0, None) == -1
    assert L.ludax_env_create(ctypes.byref(h), 11, ctypes.byref(p), 16, 0, None) == -2      # bad game
    bad = ludax.ludax_board_params(7, 7)
    assert L.ludax_env_create(ctypes.byref(h), 1, ctypes.byref(bad), 16, 0, None) == -3    # C4 is 6x7
    hex12 = ludax.ludax_board_params(12, 12)
    assert L.ludax_env_create(ctypes.byref(h), 3, ctypes.byref(hex12), 16, 0, None) == -3  # Hex <= 11
    assert L.ludax_env_create(ctypes.byref(h), 1, ctypes.byref(p), 0, 0, None) == -1       # no envs
    assert L.ludax_env_create(ctypes.byref(h), 1, ctypes.byref(p), 16, -1, None) == -1     # negative offset
    assert not h.value


def test_null_handles_are_rejected(L):
    assert L.ludax_reset(None, None) == -1
    assert L.ludax_step(None, None, None, None) == -1
    assert L.ludax_rollout(None, 0, 0, None, None, None, None) == -1
    assert L.ludax_sync(None, 0) == -1
    assert L.ludax_env_destroy(None) == 0
    assert L.ludax_mixed_plan_destroy(None) == 0
    assert L.ludax_rollout_mixed(None, 10, 0, 0, None, None, None, None) == -1
    assert L.ludax_mixed_plan_launch_host(None, 0, None, None, None) == -1
    assert L.ludax_mixed_plan_sync(None, None) == -1
    assert L.ludax_autotune_env_candidates(None, None, 0) == -1


def test_autotune_candidates_are_valid(L):
    from paper_2506_22609_b300 import ludax

    cands = ludax.ludax_autotune_candidates()
    assert len(cands) > 8
    for c in cands:
        assert 32 <= c.block_threads <= 512 and c.block_threads % 32 == 0
        assert c.blocks_per_sm == 0 or c.block_threads * c.blocks_per_sm <= 2048
        assert c.hex_nbr_table in (0, 1)
        # two envs per thread and part-filled warps only in one-thread-per-env launches
        assert c.envs_per_thread in (1, 2) and c.lanes_per_warp in (0, 8, 16)
        assert c.blocks_per_sm == 0 or (c.envs_per_thread == 1 and c.lanes_per_warp == 0)
        assert c.threads_per_env in (0, 1)  # the mixed kernel runs one lane per env
    assert {c.envs_per_thread for c in cands} == {1, 2} and {c.lanes_per_warp for c in cands} == {0, 8, 16}


def test_mixed_launch_shape_checked_before_touching_the_device(L):
    from paper_2506_22609_b300 import ludax

    fake = ctypes.c_void_p(1 << 20)  # never dereferenced: the shape is refused first
    for bad in [(128, 2, 2, 0, 0), (128, 0, 4, 0, 0), (128, 0, 8, 0, 0), (100, 0, 1, 0, 0), (128, 0, 1, 0, 4),
                (128, 0, 1, 0, 0, 2), (128, 2, 1, 0, 0, 1, 8), (128, 0, 1, 0, 0, 1, 4)]:
        cfg = ludax.make_cfg(*bad)
        assert L.ludax_rollout_mixed(fake, 10, 0, 0, fake, fake, ctypes.byref(cfg), None) == -1, bad


def test_binding_refuses_host_tensors(L):
    import torch

    from paper_2506_22609_b300 import ludax

    with pytest.raises(ValueError):
        ludax._ptr(torch.zeros(4))


def test_line_game_parameters_validated_on_host(L):
    from paper_2506_22609_b300 import ludax

    h = ctypes.c_void_p()
    ok = ludax.ludax_board_params(6, 7, 4, 2)
    assert L.ludax_env_create(ctypes.byref(h), 7, ctypes.byref(ludax.ludax_board_params(12, 12, 5, 0)), 4, 0, None) == -3
    assert L.ludax_env_create(ctypes.byref(h), 7, ctypes.byref(ludax.ludax_board_params(6, 7, 9, 0)), 4, 0, None) == -3
    assert L.ludax_env_create(ctypes.byref(h), 7, ctypes.byref(ludax.ludax_board_params(6, 7, 4, 8)), 4, 0, None) == -3
    # the other games take no line parameters
    assert L.ludax_env_create(ctypes.byref(h), 1, ctypes.byref(ludax.ludax_board_params(6, 7, 4, 0)), 4, 0, None) == -1
    assert not h.value and ok.line == 4
