"""CPU FP64 oracle for the multilevel RAS Newton-Krylov Peng-Robinson solver.

TEST INFRASTRUCTURE ONLY. Plain, slow and written to be checked by eye against
the paper (arXiv 2007.13966). Only ``tests/``, ``__graft_entry__.smoke()`` and
``bench.py``'s CPU-baseline / reference legs may import it; the product path
(the CUDA library and its binding) never does, and the two share no code.

Modules:
  eos            Section 2: PR cubic, a(T), b, m(omega), omega(T_br), dZ/dp
  discretization Section 2: CCFD two-point fluxes, BDF1/BDF2 residual, Jacobian
  schwarz        Section 3.1: partition, R_i^delta / R_i^0, ILU(k), AS / RAS
  multilevel     Section 3.2: interpolation orders 1-3, Galerkin coarse
                 operator, coarse solves, V-cycle / Kaskade / additive, Algorithm 1
  krylov         Section 3: right-preconditioned (flexible) GMRES(m)
  newton         Section 3: inexact Newton with cubic backtracking, time loop
"""
