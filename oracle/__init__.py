"""CPU FP64 oracle for the multipreconditioned directional-sweep Helmholtz solver.

TEST INFRASTRUCTURE ONLY.  Only the tests, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import this package.
The product library never calls it, and it shares no code with the CUDA path.

It is a plain, slow, step-by-step restatement of the method (Bootland & Rees,
"Multipreconditioning with directional sweeping methods for high-frequency
Helmholtz problems"):

* ``fem``      -- P1 finite elements for the impedance Helmholtz problem (Section 1,
                  Eq. (1a)-(1b)); system matrix A = K - k^2 M - i k M_Gamma and load vector.
* ``sweep``    -- non-overlapping strip decomposition, impedance-modified strip matrices
                  (Section 2, Eq. (4)) and the forward/backward double sweep (Eqs. (2)-(3)),
                  with every strip solve done by a pivoted banded LU (LAPACK zgbtrf/zgbtrs).
* ``mpgmres``  -- selective flexible multipreconditioned GMRES (Section 3) with the
                  selection rules of Section 4.
* ``direct``   -- global banded direct solve of A x = b (the plain definition of the answer).

Every function is FP64 / complex128.
"""
from . import fem, sweep, mpgmres, direct, solver  # noqa: F401
