"""GB300 library for the Chebyshev-filtered subspace iteration of the
orthogonalized enriched finite element (OEFE) method, arXiv 2010.09701.

The computation lives in liboefe.so (C ABI, include/oefe.h, CUDA for sm_103a);
this package is its binding. There is no CPU fallback: importing works
without a GPU, but creating a Context needs the built library and a device.

One pass of the subspace iteration over every k-point (Sec. IV), with the
vectors X[ik] as (ndof, nv) complex128 CUDA tensors:

    ctx = setup_workload(w)                       # mesh, enrichment, quadrature, k-points
    ctx.set_f64_products(F64_PAIRS)               # FP64-class work in FP32 pairs / exact digits
    ctx.build_hamiltonian(veff, STORE_F64 | STORE_BF16X6 | STORE_F64PAIR)
    ctx.filter_batched(X, degree, a, b, a0, FILTER_BF16X3 | FILTER_LAST_FP64)
    for ik in range(nk):
        ctx.orthonormalize(ik, X[ik])             # Cholesky-QR twice in the M inner product
        eps[ik] = ctx.rayleigh_ritz(ik, X[ik])    # Ritz values (host), X rotated in place
    mu, occ, e_band = occupations(eps, wk, nelectrons)
    ctx.density(X, occ, rho)                      # rho at every quadrature point

Here a, b, a0 are numbers or per-k lists: the lower end of the filtered interval (the
largest wanted Ritz value), the upper bound of the spectrum (upper_bound) and
the lowest Ritz value; FILTER_BF16X3 selects the tensor-core degrees, whose
split (two or three bf16 parts) follows the stored matrices.
"""
from .binding import (C64, C128, F32, F64, F64_NATIVE, F64_PAIRS, FILTER_BF16X3, FILTER_LAST_FP64, STORE_BF16X3,
                      STORE_BF16X6, STORE_COMPACT, STORE_F32, STORE_F64, STORE_F64PAIR,
                      Context, OefeError,
                      SIGNATURES, launch_count, load, occupations)
from .problem import setup_workload

__all__ = ["Context", "OefeError", "load", "launch_count", "occupations", "setup_workload", "SIGNATURES", "F64", "F32", "C128", "C64",
           "STORE_F64", "STORE_F32", "STORE_BF16X3", "STORE_BF16X6", "STORE_F64PAIR", "STORE_COMPACT", "F64_NATIVE", "F64_PAIRS",
           "FILTER_LAST_FP64",
           "FILTER_BF16X3"]
