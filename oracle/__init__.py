"""FP64 CPU oracle of the coarse-grid incremental pressure-projection step.

TEST INFRASTRUCTURE ONLY.  This package is a plain, slow restatement of the
paper's method (Kashefi, "A coarse-grid incremental pressure-projection method
for accelerating low Reynolds-number incompressible flow simulations",
Sections 2.1-2.3, Eqs. 5-27) used to check the CUDA library.  Only the test
suite, the smoke check and the CPU-baseline leg of the benchmark may import it;
the library never does, and the oracle never imports the library.

Everything is numpy/scipy in float64.  Linear systems are solved with a sparse
direct factorisation (scipy's SuperLU), so each oracle solve is the exact
discrete solution up to rounding, not an iteration stopped at a tolerance.

Modules
-------
mesh    nested hierarchy by uniform 1->4 refinement (Section 2.2) and the
        vertex-adjacency (CSR) pattern of each level.
fem     P1 element matrices M, K, Cx, Cy and the convection matrix N(w)
        (Section 2.1, Eqs. 17-20); injection and linear prolongation (Eqs. 22, 24).
flows   boundary data, forcing and closed-form solutions (Eqs. 28-30 and the
        workloads' problem statements).
cgp     the time step, Eqs. 21-26, standard (chi=0) and rotational (chi=1).
norms   discrete error norms used in the accuracy tables (Tables 1-3).
mlp     the learned initial guess network (forward / backward / Adam), float64.

Readings of points the paper leaves open are listed in the design notes and
repeated in the docstrings where they are used.  Parity status of every
function is pinned by ``tests/test_oracle_*.py``.
"""
