"""CPU oracle for the Swendsen-Wang sweep (test infrastructure only).

The oracle is a plain single-threaded C implementation (sw_oracle.c) of
Komura & Okabe, arXiv:1202.0635, Sec. 2 (Potts, Eq. 1, steps (i)-(viii))
and Sec. 4 (clock model with embedded clusters, Eq. M^2 measurement).
Only the tests, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import it.  It shares no code with the CUDA path.
"""
from .oracle import (Oracle, philox4x32_10, threshold_from_x, ncounters, observables, correlations,  # noqa: F401
                     POTTS, CLOCK, ISING)
