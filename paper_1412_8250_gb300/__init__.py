"""GB300-native periodic orbital-free DFT with higher-order finite differences.

The computation lives in libof.so (CUDA for sm_103a, C ABI in include/of.h); the module
``binding`` exposes its entry points, ``functionals`` the kinetic functionals of the paper,
``workloads`` the seeded synthetic inputs.  Importing the package loads nothing; the CUDA
library is loaded on first use of ``binding``.
"""
__all__ = ["binding", "functionals", "workloads", "build_lib"]
