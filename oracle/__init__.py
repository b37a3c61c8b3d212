"""CPU FP64 oracle for the second-order polarization-propagator window solve.

TEST INFRASTRUCTURE ONLY.  Nothing in the product path imports this package:
only ``tests/``, ``__graft_entry__.smoke()`` and the ``cpu_baseline`` /
``--impl reference`` legs of ``bench.py`` may use it.  It shares no code with
the CUDA library.

* ``pp_oracle``  dense assembly of S, A, B (orders 0, 1, 2), a matrix-free
  sigma written term by term, the dense generalized eigensolve, window
  selection and oscillator strengths.
* ``fock``       a Jordan-Wigner Fock-space brute force that evaluates the
  defining expectation values directly (no Wick algebra) and pins the closed
  forms used by ``pp_oracle`` on tiny systems.
"""

from . import pp_oracle  # noqa: F401
from . import fock  # noqa: F401
