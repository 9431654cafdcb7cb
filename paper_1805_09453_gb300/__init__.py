"""GB300-native G-prox PDHG (arXiv 1805.09453): ROF and L1-EMD solvers.

The compute path is the CUDA library built from ``csrc/`` (C ABI in
``include/gprox.h``); ``gprox`` is its Python binding and ``synth`` holds the
seeded input generators.  Importing the package does not load the library;
the first call into ``gprox`` does, and fails loudly if it was not built.
"""
__all__ = ["gprox", "synth", "build"]
