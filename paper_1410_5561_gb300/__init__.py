"""GB300-native temporally blocked 3D stencil sweeps (arXiv:1410.5561).

Submodules:
  inputs   seeded synthetic inputs (no stencil arithmetic)
  build    in-tree nvcc build of the CUDA library
  _lib     ctypes binding of include/stencil_gb300.h
  stencil  Stencil: one grid, torch tensors as device memory
  model    cache-block-size and code-balance models (Eqs. 2-5), tuner pruning
"""

__all__ = ["inputs", "build", "stencil", "model"]
