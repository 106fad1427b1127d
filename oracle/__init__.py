"""CPU oracle of the steady state-of-charge solver (test infrastructure only).

Importable from ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py``'s CPU-baseline
leg only; the CUDA library never uses it.
"""
