"""Independent FP64 CPU oracle for the FMM-preconditioned Helmholtz solver.

TEST INFRASTRUCTURE ONLY.  Nothing in the product path imports this package:
only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may use it.  It shares no code with the CUDA library; its only
shared input is the seeded workload module ``paper_1608_02461_gb300.inputs``.

Plain, slow, obviously correct numpy/scipy code in float64 / complex128.
Every function cites the part of the paper (Ibeid, Yokota, Keyes, "A
Matrix-free Preconditioner for the Helmholtz Equation based on the Fast
Multipole Method") it follows.  Where the paper is silent the reading taken is
named in the docstring (S*, B*, T*, F*, G*, D* readings).

Modules
  special      spherical Bessel/Hankel functions, spherical harmonics, Gaunt
               integrals (library routines + quadrature)
  geometry     interior nodes and constant boundary elements
  tree         uniform octree, near lists and M2L interaction lists
  translations M2M / M2L / L2L operators (exact re-expansion, then truncation)
  fmm          P2M, M2M, M2L, L2L, L2P, P2P, self terms, direct sum
  bem          the BEM-coupled FMM preconditioner (Passes A, B, C)
  tangent      exact d/dk of the truncated FMM (every stage by the product rule)
  dirichlet    inhomogeneous Dirichlet data: double-layer kernel and sums
               (direct and dipole FMM), the FDM lift, the BEM solve with data
  fdm          the 7-point finite-difference Helmholtz operator
  gmres        flexible right-preconditioned restarted GMRES

Parity status: every function is pinned by ``tests/test_oracle_*.py`` to
closed forms, library routines, brute force or convergence in p, except the
paper's 2D iteration counts, which are parity unpinned for this 3D FDM build
(context only).
"""
