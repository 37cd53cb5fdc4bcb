"""GB300-native Multigrid Monte Carlo sampler (arXiv 2407.12149).

Submodules:
  inputs -- seeded synthetic problem generators (no sampler arithmetic)
  build  -- nvcc build of libmgmc.so for sm_103a
  mgmc   -- ctypes binding of the C ABI in include/mgmc.h

The CUDA library is loaded only when mgmc.load() (or a Sampler) is used.
"""
__all__ = ["inputs", "build", "mgmc"]
