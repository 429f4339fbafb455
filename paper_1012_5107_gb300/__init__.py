"""GB300 (sm_103a) renderer for Newtonian ray tracing of the conformal grating
cloak (Halimeh, Schmied & Wegener, Opt. Express 2010).

Submodules:
  rt      -- binding of the C ABI (include/rt.h); loads libgratingrt.so
  inputs  -- seeded synthetic scenes, textures and pixel subsets
  build   -- nvcc build of the CUDA library

Importing the package does not load the CUDA library; ``rt`` does on first use.
"""
__version__ = "0.1.0"
