"""FP64 CPU oracle for the neural-preconditioned 3D-1D coupled solve.

TEST INFRASTRUCTURE.  This package is the plain, slow, obviously-correct
restatement of what the paper's method computes, written from the paper's
equations and kept independent of the CUDA path (it shares no code, constant
table or helper with ``paper_2505_08491_gb300``; only the seeded input
generators in ``mdgen`` serve both).  Only ``tests/``,
``__graft_entry__.smoke()`` and the CPU-baseline leg of ``bench.py`` may import
it.  The product path never calls it.

Modules
    fem      -- finite-element assembly of eq. (mainsys) in CSR (Section 2.1)
    cnn      -- the convolutional preconditioner network, forward and backward
                (Section 4.2, the convolution of Section 4.2's definition)
    solvers  -- sparse direct, Jacobi-CG, flexible GMRES (Section 4), the
                block-triangular preconditioner of eq. (twosteps)

Every function cites the passage it follows.  Functions whose result is not
pinned by an independent check say "parity unpinned" in their docstring.
"""
from . import fem, cnn, solvers  # noqa: F401
