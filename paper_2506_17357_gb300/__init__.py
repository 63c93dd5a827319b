"""GB300-native best-improvement VRP local search (TGA hot path).

Submodules:
  instances -- seeded synthetic instances and initial solutions (inputs only)
  tga       -- ctypes binding of libtga.so (include/tga.h), the CUDA path
  serving   -- continuous-batching request loop over the C-ABI
Building: ``paper_2506_17357_gb300.build.build()`` compiles libtga.so for sm_103a.
"""
__all__ = ["instances", "tga"]
