"""CPU oracle for the Ludax hot path -- TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  The product path (the CUDA library and
its Python binding in ``paper_2506_22609_b300``) never imports, links or runs
anything here, and nothing here imports the product package.

Contents:
  ludax_oracle.c  plain C game rules over int8 cell arrays (App. C of the
                  paper), splitmix64 draws, perft, Tic-Tac-Toe enumeration,
                  Hex connectivity by breadth-first search.
  games.py        ctypes wrapper for ludax_oracle.c (numpy in / numpy out).
  mlp.py          fp64 numpy value-network reference (forward, backward, Adam).
"""
