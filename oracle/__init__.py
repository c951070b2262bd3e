"""FP64 CPU oracle for the multi-frequency Laplace-domain elastodynamic BEM
operator (3D-ACA accelerated gCQ time-domain BEM).

TEST INFRASTRUCTURE ONLY.  Nothing in the product path imports, calls or
executes this package: only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may use it.  It shares no code with the
CUDA library (``paper_2607_15292_b300``); both sides take their inputs from
the seeded generators in ``synthetic``.

Every function is a plain, slow, FP64 restatement of the method: the
definition written out where one exists (kernels, matrix entries, dense
apply, DFT), otherwise the algorithm's steps in the paper's order (3D-ACA of
Algorithm 1, matrix-valued ACA).  Library primitives (numpy matmul, SVD, QR,
eigh, solve) serve as single steps.  Each module cites the passage it
follows.

Pins (tests/test_oracle_*.py, marked ``not gpu``) tie each function to
something other than itself: closed forms, the static Kelvin solution, the
Laplace-domain Navier residual by finite differences, rigid-body identities,
polynomial exactness, brute force on tiny inputs, the closed-form response
of a sphere under pressure, and CQ of scalar transforms with known inverse.
Functions with no such pin say "parity unpinned" in their docstring.
"""
