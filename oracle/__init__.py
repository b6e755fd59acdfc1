"""FP64 CPU oracle for PARSDMM (arXiv:1902.09699) -- TEST INFRASTRUCTURE ONLY.

This package is a plain, slow, obviously correct restatement of what the
paper's method computes, written in numpy float64.  It exists to check the
CUDA library against the paper.  Only the test suite, ``__graft_entry__.smoke``
and the ``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import
it.  The product path (the C-ABI library and its Python binding) never calls
it and shares no code with it.

Modules
-------
operators  -- grid layout and the linear operators A_i (identity, forward
              differences D_z, D_x, D_y, anisotropic TV stack), their
              adjoints, and the system matrix C (Sec. "Notation", Eq. FD_mat;
              Eq. sys_mat; set table).
prox       -- projections onto the simple sets C_i (bounds, l1 ball, l2 ball,
              cardinality) and the prox of the squared distance (Eq.
              prox_sq_dist; set table).
parsdmm    -- conjugate gradient on the normal equations, Algorithm PARSDMM,
              Algorithm adapt-rho-gamma, the feasibility / evolution stopping
              quantities (Eqs. feas_stop, obj_stop, stopping_conditions) and
              Algorithm ML-PARSDMM with its restriction / prolongation.
dykstra    -- Algorithm Parallel-DYKSTRA (Appendix A), used only as an
              independent cross-check of the PARSDMM fixed point.

Readings of places where the paper is silent or garbled are stated in the
docstring of the function that takes them.  Parity status of every function:
pinned by the tests under ``tests/test_oracle_*.py`` except where a docstring
says "parity unpinned".
"""
