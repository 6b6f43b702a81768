"""GPU-First runtime for GB300 (sm_103a): legacy-style programs run whole on one GPU.

Submodules:
  gf      -- ctypes binding of the C ABI in include/gf.h (loads libgf.so; raises if it is missing)
  inputs  -- seeded synthetic inputs (SplitMix64), shared as data by the oracle and the GPU path
  build   -- compiles the CUDA runtime and programs for sm_103a
"""
