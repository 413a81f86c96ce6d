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
forms, library routines, brute force and exact invariants; tests/test_oracle_mutations.py
plants plausible mistakes and checks that the pins catch them; tests/test_oracle_probe.py pins
the amplitude scale as well (on a noiseless periodic forward model classical and live WDD return
the object itself, unit scale included) and the probe reconstruction of Sect. 10.  The
reconstruction quality of the Hermite-Gauss bases against ground truth has no independent pin.
"""
from .wdd_oracle import *  # noqa: F401,F403
