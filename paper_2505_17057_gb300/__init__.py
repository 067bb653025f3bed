"""GB300-native explicit MMFD solver library (arXiv 2505.17057).

Submodules:
  mmfd    -- ctypes binding of the C ABI in include/mmfd.h (loads libmmfd.so; no CPU fallback)
  inputs  -- seeded synthetic initial fields (no MMFD arithmetic)
  build   -- in-tree nvcc build of libmmfd.so for sm_103a
  configs -- the benchmark / test workloads

Importing the package itself loads nothing; ``from paper_2505_17057_gb300 import mmfd``
loads the CUDA library and raises if it has not been built.
"""
