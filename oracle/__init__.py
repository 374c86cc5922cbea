"""CPU FP64 oracle of the Helmholtz FWI misfit and adjoint-state gradient.

TEST INFRASTRUCTURE ONLY: the plain, slow reference the GPU library is checked
against.  Only tests/, __graft_entry__.smoke() and bench.py's CPU-baseline leg
may import it.  It shares no code with the CUDA path and never imports it.

Parity status of each function (pins live in tests/test_oracle.py):
  helmholtz_matrix, axis_coefficients   pinned (Dirichlet eigenpairs, pointwise
                                         rebuild, Green's functions 2D/3D)
  extend, extend_adjoint                 pinned (adjoint pair, multiplicities,
                                         FD on boundary-supported directions)
  source_fields, sample_receivers       pinned (Green's function placement,
                                         hand-computed misfit)
  DirectSolver, gmres, GmresSolver      pinned (dense solve, explicit H^H)
  forward, adjoint, misfit, misfit_and_gradient
                                         pinned (zero misfit at the true model,
                                         central differences, Taylor slopes)
  prolongation, restriction             pinned (linear reproduction, 2^-d P^T)
"""
