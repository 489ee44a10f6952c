"""GB300-native direct-summation N-body library (NBSymple's method).

Submodules:
  ics    -- seeded synthetic initial conditions (numpy only)
  nbsym  -- ctypes binding of the CUDA C-ABI library ``libnbsym.so``
  build  -- compiles the CUDA library for sm_103a

Importing this package loads nothing; ``from paper_1003_3896_gb300 import
nbsym`` loads the CUDA library and raises if it has not been built.
"""
__all__ = ["ics", "nbsym", "build"]
