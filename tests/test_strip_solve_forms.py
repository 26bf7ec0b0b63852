"""The reorganised strip solves of the GPU sweep, checked on the CPU in exact-arithmetic form
(FP64 dense blocks from the oracle's matrix, tiny sizes): the recurrences that the sweep's
programs are built from give the strip solve D^{-1} r of Section 2's block LU.

* twisted block factorisation of the strip matrix T of lines 0..R-1 (line 0 absorbing, the
  rest interior): top factors F_j, bottom factors G_j, the meeting block M at q = R // 2;
* the last strip's extra line R added by the Schur complement of lines 0..R-1 after the
  first-line correction (x_R = F_R (r_R - L v[R-1]), x_j = v[j] - Z_j x_R);
* the whole last strip with its first-line coupling to the strip before it.

These are statements about the algebra only; the GPU tests compare the kernels with the
oracle's sweeps.
"""
import numpy as np
import pytest

from oracle import fem


def _blocks(k, n):
    A = fem.global_system(k, n)[0].tocsr()
    m = n + 1
    blk = lambda a, b: A[a * m:(a + 1) * m, b * m:(b + 1) * m].toarray()
    # line types of a strip: line 0 absorbing (the domain's first line), interior lines, and
    # the domain's last line for the last strip's extra line
    return blk(0, 0), blk(1, 1), blk(n, n), blk(1, 0), blk(0, 1), m


def _strip(Dbot, Dint, L, U, R, Dtop=None):
    m = Dbot.shape[0]
    lines = R + (1 if Dtop is not None else 0)
    T = np.zeros((lines * m, lines * m), dtype=complex)
    for j in range(lines):
        D = Dbot if j == 0 else (Dtop if (Dtop is not None and j == R) else Dint)
        T[j * m:(j + 1) * m, j * m:(j + 1) * m] = D
        if j > 0:
            T[j * m:(j + 1) * m, (j - 1) * m:j * m] = L
            T[(j - 1) * m:j * m, j * m:(j + 1) * m] = U
    return T


def _twisted_solve(Dbot, Dint, L, U, R, r):
    """T^{-1} r by the twisted factorisation, in the order of the sweep program."""
    q = R // 2
    inv = np.linalg.inv
    F = [inv(Dbot)]
    for j in range(1, R):
        F.append(inv(Dint - L @ F[-1] @ U))
    G = {R - 1: inv(Dint)}
    for j in range(R - 2, q, -1):
        G[j] = inv(Dint - U @ G[j + 1] @ L)
    M = inv(Dint - L @ F[q - 1] @ U - U @ G[q + 1] @ L)
    V = [None] * R
    for i in range(max(q, R - 1 - q)):        # both ends in one step
        if i < q:
            V[i] = F[i] @ (r[i] - (L @ V[i - 1] if i > 0 else 0))
        j = R - 1 - i
        if j > q:
            V[j] = G[j] @ (r[j] - (U @ V[j + 1] if j < R - 1 else 0))
    V[q] = M @ (r[q] - L @ V[q - 1] - U @ V[q + 1])
    for i in range(max(q, R - 1 - q)):
        j = q - 1 - i
        if j >= 0:
            V[j] = V[j] - F[j] @ (U @ V[j + 1])
        j = q + 1 + i
        if j <= R - 1:
            V[j] = V[j] - G[j] @ (L @ V[j - 1])
    return V, F


@pytest.mark.parametrize("k,n,R", [(20.0, 32, 8), (15.0, 40, 5), (30.0, 48, 6), (12.0, 24, 4)])
def test_twisted_solve_equals_strip_solve(k, n, R):
    Dbot, Dint, Dtop, L, U, m = _blocks(k, n)
    rng = np.random.default_rng(3)
    r = [rng.standard_normal((m, 2)) + 1j * rng.standard_normal((m, 2)) for _ in range(R)]
    V, _ = _twisted_solve(Dbot, Dint, L, U, R, r)
    T = _strip(Dbot, Dint, L, U, R)
    ref = np.linalg.solve(T, np.vstack(r))
    assert np.linalg.norm(np.vstack(V) - ref) < 1e-10 * np.linalg.norm(ref)


@pytest.mark.parametrize("k,n,R", [(20.0, 32, 8), (15.0, 40, 5)])
def test_last_strip_by_schur_complement(k, n, R):
    """The last strip (R + 1 lines, its line R of the domain's last type) with the coupling
    -L t of its line 0 to the strip before: the twisted solve of its first R lines, the
    first-line correction with Y_j = T^{-1}[j, 0] L, the line R by F_R, the correction with
    Z_j = T^{-1}[j, R-1] U.  Equals the direct solve of the bordered strip."""
    Dbot, Dint, Dtop, L, U, m = _blocks(k, n)
    rng = np.random.default_rng(5)
    r = [rng.standard_normal((m, 2)) + 1j * rng.standard_normal((m, 2)) for _ in range(R + 1)]
    t = rng.standard_normal((m, 2)) + 1j * rng.standard_normal((m, 2))
    T = _strip(Dbot, Dint, L, U, R)
    Tl = _strip(Dbot, Dint, L, U, R, Dtop)
    rhs = np.vstack(r)
    rhs[:m] -= L @ t
    ref = np.linalg.solve(Tl, rhs)

    w, F = _twisted_solve(Dbot, Dint, L, U, R, r[:R])
    Tinv = np.linalg.inv(T)
    Y = [Tinv[j * m:(j + 1) * m, :m] @ L for j in range(R)]
    Z = [Tinv[j * m:(j + 1) * m, (R - 1) * m:R * m] @ U for j in range(R)]
    v = [w[j] - Y[j] @ t for j in range(R)]                        # F3, as for every strip
    FR = np.linalg.inv(Dtop - L @ F[R - 1] @ U)                     # block Thomas's F_R
    xR = FR @ (r[R] - L @ v[R - 1])                                 # the extra line
    x = [v[j] - Z[j] @ xR for j in range(R)] + [xR]                 # the narrow corrections
    assert np.linalg.norm(np.vstack(x) - ref) < 1e-10 * np.linalg.norm(ref)
