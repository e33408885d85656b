"""GB300-native Chebyshev-filtered subspace iteration for FE spinor Kohn-Sham
Hamiltonians with noncollinear magnetism and spin-orbit coupling.

The compute path is the CUDA library ``libgbchfsi.so`` (C ABI in
``include/gbchfsi.h``); ``gbchfsi`` is its thin ctypes binding.
"""
from .gbchfsi import (BF16X3, FP32, FP64, TF32, Batch, Context, GbcError, EXPORTS,  # noqa: F401
                      LIB_PATH, alu_peak, build_info, check_selftest, fermi_occupations,
                      load_library)

__all__ = ["Context", "Batch", "GbcError", "FP64", "FP32", "TF32", "BF16X3", "EXPORTS", "LIB_PATH",
           "load_library", "fermi_occupations", "alu_peak", "build_info", "check_selftest"]
