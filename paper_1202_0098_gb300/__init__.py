"""GB300-native multiple Arnoldi method (Hoshi et al., arXiv:1202.0098).

The compute path is the in-tree CUDA library ``_build/libmka.so`` (C ABI in
``include/mka.h``); ``mka`` is its ctypes binding with the same entry-point
names.
"""
from . import build, mka

__all__ = ["build", "mka"]
