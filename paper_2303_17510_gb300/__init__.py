"""GB300-native hybrid-dealiased FFT convolutions (Murasko & Bowman, arXiv 2303.17510).

The computation lives in libhd.so (hand-written CUDA for sm_103a behind the C
ABI of include/hd.h); this package is its thin Python binding.
"""
from ._binding import (DTYPE, KIND, MULT, HdError, Plan, dealias_bound, derive_params, lib, status_string)

__all__ = ["DTYPE", "KIND", "MULT", "HdError", "Plan", "dealias_bound", "derive_params", "lib", "status_string"]
