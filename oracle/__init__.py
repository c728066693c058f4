"""FP64 CPU oracle of the lattice Boltzmann update (test infrastructure only).

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` import this package.  The product library never does.
"""
