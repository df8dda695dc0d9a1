"""GB300-native fused feature extraction (arXiv 1304.3992's data-parallel path).

The product is libfx.so (C ABI in include/fx.h, CUDA kernels for sm_103a under
csrc/); ``fx`` is its thin ctypes binding and ``build`` compiles it in-tree.
Importing this package loads nothing; ``fx.load()`` does, and raises when the
library has not been built.
"""
