"""CPU FP64 oracle for the low-rank Poisson solver (TEST INFRASTRUCTURE ONLY).

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline / reference
legs of ``bench.py`` may import this package.  The GPU product path never
imports, links or executes anything here, and nothing here imports the GPU
package: the two share no code.  Inputs come from the separate ``lrp_inputs``
module.

Contents
  poisson      -- eigenpairs of T, the orthonormal DST-I (Sec. 3), the full-grid
                  solve (Sec. 3.1), the exact spectral solution (Eq. g_for_p)
                  and error measures for low-rank results.
  cross_deim   -- scross (Algorithm "scross"), (Q)DEIM and leverage-score index
                  selection, and the adaptive Cross-DEIM loop, applied to the
                  spectral Poisson solution (Sec. 3.2).
  refine       -- the low-rank residual of a trial solution and one step of
                  iterative refinement (an extension beyond the paper; the
                  residual is the plain definition T W + W T - h^2 F).

Parity status: every function is pinned by tests in ``tests/test_oracle_*.py``
against closed forms, textbook routines or brute force (see each docstring).
"""
