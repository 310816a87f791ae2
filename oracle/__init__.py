"""FP64 CPU oracle for the IFE-CGP pressure-correction time step (test infrastructure).

This package is TEST INFRASTRUCTURE. It is a plain, slow, obviously-correct CPU restatement of
the method of Kashefi & Staples, "A Finite-Element Coarse-Grid Projection Method" (the paper's
Sect. 2.1-2.2, Eqs. 16-23 and 29-30). Only the test-suite, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import it. The CUDA library never
calls it, and it shares no code with the CUDA library (only the seeded input generators in
``cgp_inputs`` serve both).

Modules
-------
``refine``  nested 1:4 refinement and the s^p / s^u mapping tables (Sect. 2.2, Eqs. 29-30).
``fem``     closed-form P1 element matrices and global assembly (Eqs. 16-18).
``cgp``     the five-step IFE-CGP time step (Eqs. 19-23) with direct sparse solves, plus the
            Galerkin restriction and the incremental / rotational forms (options, Sect. 4) and
            an exact-projection test device (levels 0) that pins steps 2-5 by the discrete
            divergence it must remove.
``diagnostics``  body forces (drag, lift), wall shear, reattachment length and Strouhal number
            of the benchmark flows (Sect. 3.2-3.3).

Every linear system is solved by a sparse direct LU (SuperLU through ``scipy``), so the oracle's
results carry only rounding error; the CUDA path's Krylov solvers are compared against it within
their stated tolerance.

Parity status: every function here is pinned by the ``-m "not gpu"`` tests in ``tests/`` (closed
forms, invariants, brute-force quadrature on tiny meshes, convergence rates, the mesh and mapping
counts the paper prints). None is unpinned.
"""
