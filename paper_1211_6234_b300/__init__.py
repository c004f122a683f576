"""B300-native dipolar Heisenberg Monte Carlo sweep (arXiv:1211.6234).

The compute path lives in the CUDA library ``libdipmc.so`` (C-ABI declared in
``include/dipmc.h``); :mod:`paper_1211_6234_b300.dipmc` is its thin Python
binding.  Importing this package loads nothing; the binding loads the library on
first use and raises if it is missing.
"""
__all__ = ["dipmc", "inputs"]
