"""Plain, slow, CPU FP64 oracle for the matrix-free two-level deflation +
CSLP-preconditioned Krylov solver of Chen, Dwarka and Vuik (arXiv 2308.06152).

TEST INFRASTRUCTURE ONLY.  Nothing in the product path imports this package:
only ``tests/``, ``__graft_entry__.smoke()`` and the ``cpu_baseline`` /
``--impl reference`` legs of ``bench.py`` may use it.  It shares no code with
the CUDA library (no kernels, headers, tables or helpers); the two meet only
through the seeded input arrays the tests hand to both.

Every operator is assembled as a SciPy CSR matrix over the *unknowns* of a
grid level (all nodes under Sommerfeld boundaries, interior nodes under
homogeneous Dirichlet boundaries) and every product is a sparse mat-vec.
Vectors handed in or out of the public functions are full grids of shape
``(ny, nx)`` (x fastest), complex128, with zeros on Dirichlet boundary nodes.

Modules
-------
operators  -- grid hierarchy, Helmholtz / CSLP matrices, transfer operators,
              deflation vectors and the coarse operators E (Sec. 2, 3, 5).
krylov     -- GMRES with modified Gram-Schmidt and Givens rotations
              (Algorithm 1), right-preconditioned, flexible and left-
              preconditioned forms.
solver     -- multigrid V-cycle for the CSLP, inner coarse solve, A-DEF1
              preconditioner and the outer flexible GMRES (Sec. 3, 5, 6).
gradient   -- adjoint misfit gradient with respect to squared slowness.

Scripts: ``record_bench_counts`` writes the oracle's iteration counts for
the benchmark workloads (scales the CPU baseline); ``paper_tables`` prints
the oracle's outer counts beside those printed in Tables 2, 3 and 5 (and
Table 5's inner counts).

Parity status: every function is pinned by a ``-m "not gpu"`` test in
``tests/test_oracle_*.py``.  The corner ghost value of the ReD-Glk2
boundary rule, which the paper leaves open, is pinned by consistency (the
corner-adjacent rows converge like H^2 on a smooth function satisfying the
Sommerfeld condition); Table 5's inner iteration counts are pinned at the
coarse tolerance of the convergence study (1e-12).
"""

from . import operators, krylov, solver, gradient  # noqa: F401
