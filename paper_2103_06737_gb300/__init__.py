"""GB300 (sm_103a) charge-conserving FEM-PIC hot path of arXiv 2103.06737.

Submodules:
  fem_pic  -- Python binding of the C ABI (include/fem_pic.h) over libfempic.so
  build    -- nvcc build of the library (in-tree, sm_103a)
  inputs   -- seeded synthetic meshes, particles and field DOFs
"""
