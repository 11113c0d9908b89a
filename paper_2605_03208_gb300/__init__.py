"""GB300-native snapshot digest, dedup, pointer census, restore and compare.

The compute path is the CUDA library ``libkc.so`` (sources in ``csrc/``,
C ABI in ``include/kc.h``); ``kc`` is its Python binding.
"""
from . import build, kc, workloads  # noqa: F401

__all__ = ["build", "kc", "workloads"]
