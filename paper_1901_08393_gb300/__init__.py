"""GB300-native dense P0 single-layer BEM capacity library (arXiv 1901.08393 hot path).

``bem`` is the ctypes binding of the CUDA library (C ABI in include/bem.h);
``inputs`` builds the seeded synthetic meshes; ``build`` compiles the library.
"""
