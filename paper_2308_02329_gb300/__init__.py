"""GB300-native simulator of the coherent hyperspin machine (arXiv 2308.02329).

The compute path lives in the CUDA library built from ``csrc/`` and is reached
through the C ABI declared in ``include/chym.h``; ``chym`` is the thin ctypes
binding.  Importing this package loads nothing: the native library is loaded on
first use and a missing library is an error, never a fallback.
"""
__all__ = ["chym", "inputs"]
