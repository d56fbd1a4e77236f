"""ffsyrk: C = A·Aᵀ over a prime field on one GB300 (arXiv 2001.04109, Algorithm 2).

The compute path is the C-ABI CUDA library built from ``csrc/`` (see
``include/ffsyrk.h``); :mod:`paper_2001_04109_gb300.ffsyrk` is its ctypes
binding.  Importing this package loads nothing: the binding loads the
library on first use and raises if it is missing.
"""
__version__ = "0.1.0"
