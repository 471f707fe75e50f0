"""GB300 library for the Chebyshev-filtered subspace iteration of the
orthogonalized enriched finite element (OEFE) method, arXiv 2010.09701.

The computation lives in liboefe.so (C ABI, include/oefe.h, CUDA for sm_103a);
this package is its binding. There is no CPU fallback: importing works
without a GPU, but creating a Context needs the built library and a device.
"""
from .binding import (C64, C128, F32, F64, F64_NATIVE, F64_PAIRS, FILTER_BF16X3, FILTER_LAST_FP64, STORE_BF16X3,
                      STORE_BF16X6, STORE_F32, STORE_F64, STORE_F64PAIR,
                      Context, OefeError,
                      SIGNATURES, launch_count, load, occupations)
from .problem import setup_workload

__all__ = ["Context", "OefeError", "load", "launch_count", "occupations", "setup_workload", "SIGNATURES", "F64", "F32", "C128", "C64",
           "STORE_F64", "STORE_F32", "STORE_BF16X3", "STORE_BF16X6", "STORE_F64PAIR", "F64_NATIVE", "F64_PAIRS",
           "FILTER_LAST_FP64",
           "FILTER_BF16X3"]
