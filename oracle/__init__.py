"""Plain CPU FP64 oracle of the orthogonalized enriched finite element (OEFE)
Chebyshev-filtered subspace iteration (Rufus, Kanungo, Gavini, arXiv 2010.09701).

TEST INFRASTRUCTURE ONLY. This package is the slow, obviously correct
restatement of the paper's definitions that the CUDA library is checked
against. Only the tests, ``__graft_entry__.smoke()`` and the CPU-baseline leg
of ``bench.py`` may import it. It shares no code with the CUDA library and the
library never calls it.

Every function states the passage it follows: "Eq. X" is an equation label of
the paper, "Sec. III" a section. Where the paper is silent the reading taken is
stated in the function's docstring.

Modules
-------
fe1d        1D GLL and Gauss rules, Lagrange basis on GLL nodes
mesh        periodic rectilinear spectral-element mesh, lumped GLL mass
quadrature  per-cell point sets (plain, enriched, octree toward nuclei)
adaptive    convergence-driven adaptive point sets (trial integrals per box)
enrichment  truncated atomic orbitals, smooth cutoff, Bloch phase, supports
operators   cell Hamiltonians, orthogonalizing coefficients, overlap blocks
solver      Chebyshev filter, Cholesky-QR, Rayleigh-Ritz, occupations,
            density, band energy, adjoint, residuals
electrostatics  smeared nuclear charges, their potential, the periodic Poisson
            solve, the nuclear correction, the electrostatic energy
xc          LDA exchange and correlation (Ceperley-Alder data, Perdew-Zunger fit)
mixing      linear and Anderson density mixing
scf         the self-consistent field loop and the total energy
"""
