"""GB300-native SDMM-SARA radio-interferometric imaging (arXiv:1307.4370).

The compute path is the CUDA library built from ``csrc/`` (C ABI in
``include/purify.h``); ``binding`` is its thin ctypes binding, ``inputs`` the
seeded synthetic-input generator.  Importing the package loads nothing; the
library is loaded on first use and its absence is an error (no fallback).
"""

__all__ = ["binding", "inputs", "build"]
