"""GB300 state-vector simulator: the amplitude-pairing hot path of QVecOpt
(arXiv 2508.15545) as sm_103a CUDA kernels behind a C ABI (include/qv.h).

Submodules:
  workloads  seeded synthetic circuits / states (no simulation arithmetic)
  qv         ctypes binding of libqv.so, same names as the C ABI
  autograd   torch.autograd.Function around the adjoint-gradient entry point
  build      compiles libqv.so for sm_103a

Importing the package does not load the CUDA library; ``qv`` does, and raises
if it is missing.
"""
__all__ = ["workloads", "qv", "build"]
