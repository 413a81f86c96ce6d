"""FP64 CPU oracle for live Wigner Distribution Deconvolution (test infrastructure only).

This package is the plain, slow, obviously correct statement of what the GPU path computes.  It is
test infrastructure: only the test suite, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import it.  The product path never calls it, and it shares no code, tables or
helpers with the CUDA library.

Modules
  wdd_oracle  classical WDD (Eq. 2, Eq. 3), the pre-computed Wiener filter (Algorithm 1), the
              modified live WDD (Algorithm 2), the Hermite-Gauss bases (Sect. 4, Sect. 5) and the
              overlap criterion (Sect. 6.2, Eq. 15-17).

Pins: tests/test_oracle_pins.py checks every function against values the paper prints, closed
forms, library routines, brute force and exact invariants, and tests/test_oracle_mutations.py
plants plausible mistakes and checks that the pins catch them.  One quantity has no independent
pin: the absolute amplitude scale of the reconstructed object (the division by sqrt(o_0) in
``finalize``), so its parity is unpinned; only the phase is graded.
"""
from .wdd_oracle import *  # noqa: F401,F403
