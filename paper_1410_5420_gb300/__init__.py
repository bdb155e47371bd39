"""GB300-native presorting k-d tree builder (Brown, arXiv 1410.5420).

The compute path is the CUDA library ``libkdtree.so`` (C ABI in
``include/kdtree.h``); ``api`` is its Python binding with the same names.
"""
from __future__ import annotations

__all__ = ["api", "build"]
