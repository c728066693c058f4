"""GB300-native lattice Boltzmann hot path of arXiv:1202.0442 (lb2d.pm 0.1).

The library is the C ABI of ``include/lb2d.h`` implemented by the CUDA
kernels in ``csrc/``; ``lb2d`` is its Python binding and ``synth`` draws the
seeded synthetic workloads.  Importing the package loads nothing: the CUDA
library is loaded on first use and raises if it has not been built.
"""
__all__ = ["lb2d", "synth", "build"]
