"""FP64 CPU oracle for the low-memory S_N-DG method (Sun & Hauck, arXiv 1907.01027).

TEST INFRASTRUCTURE ONLY.  Nothing here is part of the product: only ``tests/``, ``__graft_entry__.smoke()``
and the CPU-baseline leg of ``bench.py`` may import it.  It shares no code with the CUDA path; both take
their inputs from :mod:`workloads`.

Two independent implementations of what the method computes:

* :mod:`oracle.dense` -- the definition written out: the global bilinear form B and functional Q_alpha of
  Section 2.1 assembled entry by entry from the Appendix A integrals (evaluated by Gauss quadrature of the
  basis functions), restricted to each variant's trial/test spaces by explicit basis matrices (Section 3.2
  low-memory space, Section 3.3 reconstructed Petrov-Galerkin space) and solved directly.  Tiny meshes.
* :mod:`oracle.sweeps` (+ ``csweep.c``) -- the paper's algorithms step by step: the block operators L, M, P,
  Sigma, B11 and R applied matrix-free, transport sweeps as block lower-triangular solves in upwind order,
  the reduced systems eq-sndg-phi / eq-lmdg-reducemat / eq-rlmdg-reducemat solved by a library Krylov
  method, and the recovery steps.  Any mesh size.
* :mod:`oracle.dsa` -- the diffusion correction of the cell averages, a right preconditioner for GMRES on the
  reduced systems (not from the paper, which leaves preconditioners to future work).
* :mod:`oracle.slab1d` -- the slab-geometry versions of the schemes (Section 4.1), assembled as trial/test
  restrictions of the 1D P1 form and solved directly: a cross-check of the scheme readings against the
  paper's printed 1D errors.

Pins (``tests/test_oracle_*.py``): quadrature moments, Appendix A integrals against closed forms, exact
reproduction of states that lie in each trial space, particle balance, B11 symmetry/definiteness,
convergence orders of Table tab-2d-aniso, the diffusion limit of Example examp-2ddifflim and the
nine-point limit stencil of Section 3.1, sweep-vs-dense agreement on tiny meshes, and the slab Tables
tab-1d-aniso and tab-1d-eps10-5.
"""
