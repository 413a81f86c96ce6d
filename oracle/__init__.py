"""FP64 CPU oracle for live Wigner Distribution Deconvolution (test infrastructure only).

This package is the plain, slow, obviously correct statement of what the GPU path computes.  It is
test infrastructure: only the test suite, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import it.  The product path never calls it, and it shares no code, tables or
helpers with the CUDA library.

Modules
  wdd_oracle  classical WDD (Eq. 2, Eq. 3), the pre-computed Wiener filter (Algorithm 1), the
              modified live WDD (Algorithm 2), the Hermite-Gauss bases (Sect. 4, Sect. 5) and the
              overlap criterion (Sect. 6.3).

Parity status of each function is given in its docstring; functions whose result has no
independent pin say "parity unpinned".
"""
from .wdd_oracle import *  # noqa: F401,F403
