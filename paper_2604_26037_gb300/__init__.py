"""GB300-native PAW finite-element Chebyshev filter (Python binding).

Thin ctypes layer over ``libpawfe.so`` (C ABI declared in include/paw_fe.h):
argument marshalling only.  Every operator application, filter step,
Rayleigh-Ritz projection and gradient runs in the library's CUDA kernels.
PyTorch supplies device memory and the current CUDA stream.  There is no
CPU fallback: importing this package fails if the library is missing.
"""
from ._lib import (PawBatch, PawError, PawFE, Precision, build_library, lib_path, load_library,
                   SubspaceEnergy)

__all__ = ["PawBatch", "PawError", "PawFE", "Precision", "build_library", "lib_path", "load_library",
           "SubspaceEnergy"]
