"""GB300-native compressed H / UH / H^2 matrix-vector products (libhm).

The compute path is the C-ABI library ``libhm`` (host construction and
packing in C++, products in hand-written sm_103a CUDA kernels); this package
only builds it and marshals arguments to it.
"""
from .hm import HMatrix, HMError  # noqa: F401

__all__ = ["HMatrix", "HMError"]
