"""B300-native doubly-periodic slab spectral Ewald solver.

The solve is the CUDA library built from csrc/ (C ABI: include/dpslab.h);
``dpslab`` is its Python binding and ``synth`` the seeded input generator.
"""
