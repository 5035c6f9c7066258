"""Plain FP64 CPU oracle for the staggered Kahler-Dirac multigrid solver.

TEST INFRASTRUCTURE.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline / reference legs of ``bench.py`` may import anything from here.
The CUDA library never calls into this package and shares no code with it;
the two meet only in the seeded input generators of
``paper_2212_12559_gb300.inputs``.

Everything is numpy complex128, written for a reader checking it against the
paper by eye rather than for speed:

* ``lattice``  -- site ordering, neighbours, staggered phases eta_mu(x), the
  chirality eps(x), Kahler-Dirac 2^4 blocks and 4^4 aggregates (Sec. 2.2).
* ``dirac``    -- the staggered operator M = m + D (naive, or with Naik long
  links), its split D = B + C into in-hypercube and between-hypercube hops
  (Eq. 1), the block inverse (B+m)^{-1} and A = (B+m)^{-1} M (Eq. 2).
* ``coarse``   -- near-null vectors by CGNE on the homogeneous system, chiral
  doubling, block orthonormalisation, R = P^dag and the Galerkin operator
  R A P stored as a 9-point stencil (Sec. 2.1, 2.3).
* ``solvers``  -- GCR, the s-step CA-GCR smoother, CGNE (Sec. 2.1, 3.2).
* ``mg``       -- the K-cycle preconditioned outer GCR (Sec. 2.1, Table 1).
* ``force``    -- the fermion action phi^dag (M^dag M)^{-1} phi and its
  derivative with respect to links and mass.

Parity pins (tests marked ``not gpu``) tie each function to facts fixed by the
paper or by mathematics: free-field closed forms, (anti/eps-)Hermiticity,
gauge covariance, dense brute force on tiny lattices and library routines.
"""
