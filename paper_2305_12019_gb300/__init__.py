"""GB300-native generalized DWD solver (inexact sGS-ADMM hot path).

The solver lives in the CUDA library ``libgdwd.so`` (C-ABI declared in
``include/gdwd.h``); :mod:`paper_2305_12019_gb300.gdwd` is its thin ctypes
binding.  Importing this package loads nothing; the binding loads the library on
first use and raises if it is missing.
"""
__all__ = ["gdwd", "synth"]
