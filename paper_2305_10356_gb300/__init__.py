"""Spectral clustering via orthogonalization-free methods on GB300 (sm_103a).

The compute path is the CUDA library libofsc.so (C ABI in include/ofsc.h); `ofsc` is its thin
binding, `synth` the seeded input generators, `build` the in-tree nvcc build.
"""
from . import ofsc  # noqa: F401
