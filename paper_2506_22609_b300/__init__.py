"""B300-native batched board-game engine (Ludax hot path, arXiv 2506.22609).

The compute path is ``libludax.so`` (hand-written sm_103a CUDA behind the
C-ABI of ``include/ludax.h``); ``ludax`` is its Python binding.
"""
__all__ = ["ludax", "workloads", "build"]
