"""GB300 (sm_103a) modal discontinuous Galerkin solver for 2D Euler.

Modules:
  dg      -- ctypes binding of the C ABI (include/dg.h); the CUDA library
             libdg.so is loaded on first use and its absence is an error.
  inputs  -- seeded synthetic meshes and initial data.
  _build  -- in-tree nvcc build of libdg.so for sm_103a.

Importing the package loads nothing; ``dg.load()`` (or any call) loads the
library.
"""
__all__ = ["dg", "inputs"]
