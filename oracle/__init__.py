"""CPU oracle for the rank-Greville recursive least-squares update (TEST INFRASTRUCTURE).

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of ``bench.py`` may
import this package. It shares no code with the CUDA library and never imports it.

  * ``oracle.fp64``    -- ctypes wrapper of ``rg_oracle.c``: plain FP64 Algorithm 1, the
                         orthonormal and orthogonal variants of Section 2.2, and the
                         pseudoinverse update of Theorems 2/3.
  * ``oracle.exact``   -- exact-rational Algorithm 1 and the Theorem 1 route (fractions).
  * ``oracle.checks``  -- Penrose conditions, invariants and the Section 4.2 metrics.
  * ``oracle.adjoint`` -- the derivative of X = A^+ y from a library pseudoinverse or from
                         the FP64 oracle's factors.
"""
