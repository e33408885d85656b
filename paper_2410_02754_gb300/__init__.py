"""GB300-native Chebyshev-filtered subspace iteration for FE spinor Kohn-Sham
Hamiltonians with noncollinear magnetism and spin-orbit coupling.

The compute path is the CUDA library ``libgbchfsi.so`` (C ABI in
``include/gbchfsi.h``); ``gbchfsi`` is its thin ctypes binding.
"""
from .gbchfsi import (FP32, FP64, Batch, Context, GbcError, EXPORTS, LIB_PATH,  # noqa: F401
                      fermi_occupations, load_library)

__all__ = ["Context", "Batch", "GbcError", "FP64", "FP32", "EXPORTS", "LIB_PATH", "load_library",
           "fermi_occupations"]
