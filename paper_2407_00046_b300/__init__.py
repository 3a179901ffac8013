"""B300-native barrier-augmented Lagrangian (arXiv 2407.00046) inexact
Newton-PCG time step.

  scenes  seeded synthetic scene generators (inputs only)
  bal     ctypes binding of libbal.so (the CUDA implementation)
  build   nvcc build of libbal.so for sm_103a
"""
__all__ = ["scenes", "bal", "build"]
