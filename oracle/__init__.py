"""Plain FP64 CPU oracle for the deflated Hutchinson estimator of Tr(A^-1).

TEST INFRASTRUCTURE ONLY.  Nothing on the product path may import, call or
execute anything in this package: only the test suite, the smoke check and
the CPU-baseline leg of the benchmark do.  The oracle shares no code with the
CUDA library; the two meet only through the seeded input generator
(``paper_1603_05988_gb300.synth``), which holds none of the method's
arithmetic.

Everything here is written for a reader checking it against the paper by eye:
explicit matrices, plain loops or single library primitives (sparse matvec,
dense LU, Hermitian eigendecomposition), FP64 throughout, no blocking or
fusion.  Each function cites the passage of Gambhir, Stathopoulos & Orginos,
"Deflation as a method of variance reduction for estimating the trace of a
matrix inverse" (SIAM J. Sci. Comput. 2017, arXiv:1603.05988) it follows.

Modules
  gamma      chiral Dirac matrices (basis reading, see module docstring)
  lattice    site indexing, coordinates, neighbours
  wilson     explicit sparse A, matrix-free A, explicit A^H
  philox     Philox4x64-10 counter-based generator (Salmon et al., SC'11)
  noise      Z4 noise z0, hierarchical-probing colouring and Hadamard vectors
  exact      exact Tr(A^-1) (LU), eq. (1.2) variance, free-field closed forms,
             Theorem 2.1, the 3x3 example of Section 2
  solve      dense LU and CGNR reference solvers
  deflation  k smallest singular triplets via dense eig of gamma5*A; T_D and
             the deflation quadrature in the paper's literal A^H form
  estimator  Algorithm 1 (deflatedHP), sample variance and the jackknife of
             the mean over z0 runs
"""

# submodules are imported explicitly by callers (from oracle import wilson, ...)
