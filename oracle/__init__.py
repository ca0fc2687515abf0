"""Oracle for the FLUPS Fourier Poisson solve (arXiv 2211.07777): plain FP64 CPU code.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` (``--impl reference`` included) may import,
call or execute anything in this package.  It shares no code, header, table or
helper with the CUDA path (``paper_2211_07777_gb300``) and imports nothing
from it; the two meet only through the seeded input generators, which hold
none of the method's arithmetic.

Parity status of each function (what pins it, see ``tests/test_oracle_*.py``):

* ``solver.extend`` / ``solver.restrict``: every symmetric, periodic, unbounded
  and semi-unbounded extension against O(N^2) sums of the paper's transform
  definitions (Section 2.2) and the textbook DCT/DST types II and IV.
* ``solver.solve`` with the spectral, HEJ2..HEJ10 and LGF2 kernels on
  symmetric/periodic BCs: the paper's printed E_inf (Section "Validation",
  symmetric and periodic case) to ~1e-12 relative.
* ``solver.solve`` fully unbounded, HEJ2 and HEJ0: the printed E_inf of the
  fully unbounded case; O(N^6) direct sums; the closed-form Gaussian-blob
  potential.
* ``green.hej2_1d`` / ``green.hej2_2d``: against adaptive quadrature of the
  heat-kernel integral and against the K0 far field.
* mixed spectral/unbounded solves: mode-by-mode 1D/2D direct convolutions.
* ``solver.biot_savart``: periodic closed form (curl of sine modes) and
  consistency with the scalar solve of each curl component.
"""
from .solver import (  # noqa: F401
    CELL, NODE, EVEN, ODD, PER, UNB, Problem, solve, biot_savart, curl_bc,
    direction_type, direction_order, extend, restrict, extended_length, green_spectrum, set_fft_workers,
)
from . import green  # noqa: F401
