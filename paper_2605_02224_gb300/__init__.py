"""GB300-native Manifold k-NN: exact batched k-NN queries over successor lists.

The compute path lives in libmknn.so (C ABI in include/mknn.h): a host
builder for the successor table and hand-written CUDA kernels for sm_103a
for the queries. This package is its ctypes binding (`mknn`) plus a small
convenience wrapper (`Cloud`). There is no CPU fallback: if the library is
missing, importing the binding's functions raises.
"""
from __future__ import annotations

from . import mknn  # noqa: F401
from .mknn import MknnError  # noqa: F401
from .cloud import Cloud  # noqa: F401

__all__ = ["mknn", "MknnError", "Cloud", "build"]


def build(verbose: bool = False) -> str:
    """Compiles libmknn.so for sm_103a in-tree and returns its path."""
    from . import _build
    return _build.build(verbose=verbose)
