"""FP64 CPU oracle for the matrix-probing hot path -- TEST INFRASTRUCTURE ONLY.

This package is a plain, slow, obviously-correct NumPy implementation of what
the GPU library computes.  It exists to check the CUDA path.  Only ``tests/``,
``__graft_entry__.smoke()`` and the CPU-baseline leg of ``bench.py`` may import
it; the product path (the ``paper_1101_3615_gb300`` package and its CUDA
library) never imports, links or calls anything here, and shares no code,
constants or tables with it.  Inputs come from the separate ``workloads``
package, which holds no method arithmetic.

Modules
-------
fd      8th-order central second-derivative weights (derived, not typed in),
        zero-extended Laplacian, absorbing-sponge profile.
wave    discrete nonlinear forward map, Born operator F (Sec. 2 equations),
        its exact transpose F* (reverse-time migration, Sec. 1.1), the normal
        operator H = F*F stacked over shots, and the misfit gradient.
symbol  elementary operators B_i of the symbol expansion (Eq. compr2), the
        randomized least-squares fit of Sec. 1.4 and the preconditioner apply.
solve   iterative solution of the linearised least-squares problem (gradient
        descent, optionally preconditioned; conjugate gradients on the normal
        equations) and the Krylov trial functions, as Sec. 2 compares them.
spectrum dense assembly of a model-space operator (brute force) and its
        epsilon-rank, the quantity Sec. 2 tabulates for its Hessian.

Parity status: every function here is pinned by a ``-m "not gpu"`` test
against closed forms, invariants or brute force (see ``tests/test_oracle_*``).
"""
