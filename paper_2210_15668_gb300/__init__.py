"""GB300 (sm_103a) TDGL + Poisson time step of FerroX (arXiv 2210.15668).

Modules:
  inputs   seeded synthetic device stacks and initial polarization (data only)
  ferrox   ctypes binding of the CUDA library libferrox (include/ferrox.h)
  build    nvcc build of the library, in-tree

Importing the package loads nothing; `ferrox.load()` (or `ferrox.Device`) loads
the compiled library and raises if it has not been built.
"""
