"""Global direct solve of A x = b: the plain definition of the discrete solution.

A in the global numbering g = j (n + 1) + i is banded with half-bandwidth n + 2 (the
north-east neighbour sits n + 2 positions away), so a pivoted banded LU (LAPACK zgbtrf /
zgbtrs) gives x = A^{-1} b.  Host memory ~ (3 (n + 2) + 1) (n + 1)^2 * 16 bytes.
"""
from __future__ import annotations

import numpy as np

from . import fem, sweep


def solve(A, b: np.ndarray, n: int) -> np.ndarray:
    bw = n + 2
    lu = sweep.BandLU(A, bw)
    return lu.solve(np.asarray(b, dtype=np.complex128))


def dense_solve(A, b: np.ndarray) -> np.ndarray:
    """Dense LU (numpy) for tiny grids."""
    return np.linalg.solve(A.toarray(), np.asarray(b, dtype=np.complex128))


def problem(k: float, n: int, sources) -> tuple:
    """(A, b) for the impedance problem with Gaussian sources (g = 0)."""
    A, K, M, MG = fem.global_system(k, n)
    b = fem.load_vector(n, M, MG, fem.gaussian_source(n, sources))
    return A, b
