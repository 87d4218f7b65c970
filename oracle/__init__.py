"""CPU oracle for the matrix-free Poisson operator of Kronbichler & Wall,
"A performance comparison of continuous and discontinuous Galerkin methods
with fast multigrid solvers" (arXiv:1611.03029).

TEST INFRASTRUCTURE ONLY.  Nothing in the product path may import this
package: only the test suite, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` use it.  It
shares no code, tables or helpers with the CUDA library in
``paper_1611_03029_gb300``; the two meet only through the vector layouts
documented in ``include/mfpoisson.h``.

The oracle is deliberately plain: it assembles the stiffness matrix element
by element from full 3D basis-function products at Gauss points (no sum
factorisation), stores it as a sparse matrix and solves with textbook
iterations, all in float64.  Every function cites the passage of the paper
it follows.

Modules
  fem      reference element, mesh and mapping (analytic maps or given
           support points), cell and SIPG face assembly,
           load vector, L2 error, Neumann / inhomogeneous Dirichlet data and
           a direct solve for manufactured solutions (Sec. 2, 2.1, 2.2;
           Eq. 4, 6, 7, 12)
  cube     the paper's three-Gaussian example on (-1, 1)^3 (Sec. 4.3), pinned
           against the L2 errors it prints
  mg       level hierarchy (coefficient and support-point coarsening),
           Jacobi diagonal, Chebyshev smoother, CG-Lanczos eigenvalue
           estimate, transfer, coarse Chebyshev solve, V-cycle, PCG (Sec. 4.1)
  adjoint  assembled coefficient derivative and dL/da (not in the paper)
  rows     sampled rows of the operator for large meshes (Eq. 12)
  hdg      hybridizable DG blocks, the statically condensed trace solve, the
           element-by-element post-processing and the mixed HDG operator
           (Sec. 2.3, Sec. 3 "HDG mixed matrix-free"), pinned against the
           HDG L2 errors the paper prints

Parity status: every function is pinned by tests in tests/test_oracle_*.py
(closed forms, invariants, printed values of the paper; the curved geometry
and the coarsening rules in test_oracle_geometry.py).
The float32 V-cycle of the mixed-precision path has no float32 oracle: it is
compared with the float64 V-cycle within a float tolerance.
"""
