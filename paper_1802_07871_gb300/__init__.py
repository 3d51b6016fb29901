"""GB300-native charge-transfer bond-order MD (arXiv:1802.07871).

The computation lives in the CUDA library libctbop.so (C ABI in
include/ctbop.h); `ctbop` is its ctypes binding and `structures` generates
seeded synthetic inputs. Importing the package does not load the library.
"""
__all__ = ["ctbop", "structures", "build"]
