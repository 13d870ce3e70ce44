"""Plain FP64 CPU oracle for the Stokes-IB multigrid solve (Bhalla, Knepley, Adams, Guy, Griffith).

TEST INFRASTRUCTURE ONLY.  This package is a slow, literal restatement of the paper's method in
numpy/scipy, written to check the CUDA path.  Only the test-suite, the smoke check of
``__graft_entry__`` and the CPU-baseline leg of ``bench.py`` may import it.  The product path
(``paper_1612_02208_gb300`` and its CUDA library) never imports, links or calls anything here,
and this package imports nothing from the product except the seeded input generators
(``paper_1612_02208_gb300.inputs``), which hold no arithmetic of the method.

Modules
  peskin    -- the four-point kernel phi and its derivative (Appendix, Lagrangian-Eulerian interaction)
  mac       -- staggered-grid Laplacian, gradient, divergence, momentum operator (Appendix, Eulerian discretization)
  ib        -- interpolation J, spreading S, spring stiffness K, S K J (Sec. 2.2, Appendix)
  system    -- Stokes-IB operator, right-hand side, gauge, three independent exact solves (Eqs. system-impib, matrix-impib)
  transfer  -- RT0 velocity prolongation, its adjoint restriction, pressure transfers (Sec. 3.2)
  smoothers -- additive Vanka (Alg. 2 as per-cell additive Schwarz) and Schur-complement smoothing (Eq. approx-fact-Stokes-IB)
  multigrid -- level hierarchy with the Galerkin coarse IB operator and the recursive V-cycle (Alg. 1)
  krylov    -- flexible GMRES with classical Gram-Schmidt twice
  adjoint   -- adjoint solve and gradients with respect to spring stiffness and marker positions

Parity status of each function is recorded in its docstring; every function is pinned by a test
in ``tests/test_oracle_*.py`` against closed forms, invariants or brute force, except where a
docstring says "parity unpinned".
"""
