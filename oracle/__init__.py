"""Plain FP64 CPU oracle of the agglomeration h-multigrid for CDG Poisson.

TEST INFRASTRUCTURE ONLY.  Only the tests, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import this package.  The GPU library never
calls it, and it shares no code with the library (the seeded input generators
in ``synthetic`` are the only common module).

Every function follows the paper (Pan & Persson, "Agglomeration-Based Geometric
Multigrid Solvers for Compact Discontinuous Galerkin Discretizations on
Unstructured Meshes") step by step, with plain loops and library primitives
(numpy / scipy.sparse products, dense solves), and cites the passage it
restates.  Readings of passages that are silent, garbled or ambiguous are
labelled R1..R16 in the docstrings.

Parity pins (tests/test_oracle_*.py): quadrature against closed-form simplex
moments; basis Gram = I; operator symmetry, SPD, polynomial reproduction,
closed-form lifting energy of piecewise constants, L2 convergence order p+1;
the C-matrix second-neighbour pattern of Section 4.2; a hand-traced
agglomeration example; coarse operators against an independent assembly route;
PCG against a dense direct solve.  Parity unpinned: the tie-break rules of the
agglomeration (R9, R10) and the choice of consistent switch (R4) have no value
in the paper to check against; they are pinned only by their written rules.
"""
