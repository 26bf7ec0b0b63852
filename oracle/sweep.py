"""Non-overlapping strip decomposition and directional double sweeps (Section 2).

Decomposition (Section 2, Figure 1; non-overlapping reading).  The node lines across the
sweep direction are split into N strips of R = n / N consecutive lines; the strip that a
sweep visits LAST owns one extra line (n + 1 = N R + 1 lines in total).  Between two
neighbouring strips lies one layer of cells that belongs to neither strip.

    BT: row strips (lines j), visited bottom -> top; top strip has R + 1 lines.
    TB: row strips, visited top -> bottom; bottom strip has R + 1 lines.
    LR: column strips (lines i), visited left -> right; rightmost strip has R + 1 lines.
    RL: column strips, visited right -> left; leftmost strip has R + 1 lines.

Impedance-modified strip matrix.  A sweep is a block LU factorisation whose Schur
complements are approximated by a transparent-condition surrogate (Section 2: forward and
backward sweeps are block forward / backward substitution, and approximate transparent
conditions are approximate Schur complements).  The exact Schur complement of strip s
is its block of A plus the discrete Dirichlet-to-Neumann map of everything already swept
(the cell layer on the swept side and all strips beyond it).  Here that map is replaced by
the zeroth-order impedance condition of Eq. (4), du/dn - i k u, on the interface facing the
swept strips.  So D_s is the P1 matrix of the strip's cells together with the cell layer on
its FAR side (towards the strips not yet visited), restricted to the strip's own nodes,
with M_Gamma on the facing interface and on the physical sides:

    D_s = A_ss - (swept-side cell layer's part of A_ss) - i k M_Gamma(facing interface).

Its far-side rows are exactly those of A.  The last strip visited has no far layer; its
far side is the physical boundary.

Double sweep (Section 2, Eqs. (2)-(3), as a forward-then-backward block Gauss-Seidel over
strips in the sweep order, with D_s as diagonal blocks and the global couplings of A
between neighbouring strips as off-diagonal blocks):

    forward:  v_s = D_s^{-1} (r_s - A_{s,prev} v_prev)              for s in sweep order
    backward: u_last = v_last  (one solve in the last strip, Section 2)
              u_s = v_s - D_s^{-1} (A_{s,next} u_next)             for s in reverse order

i.e. M = (D + L) D^{-1} (D + U) in the sweep ordering.  A single (forward-only) sweep
returns v.  Every strip solve is a pivoted banded LU (LAPACK zgbtrf / zgbtrs) of D_s in
its own line-by-line numbering (bandwidth m + 1).
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp
from scipy.linalg import lapack

from . import fem

DIRECTIONS = ("LR", "RL", "BT", "TB")


def strip_lines(n: int, N: int, direction: str) -> list[tuple[int, int]]:
    """Line ranges [a, b] (inclusive) of the strips, listed in SWEEP order."""
    if n % N != 0:
        raise ValueError("n must be a multiple of the number of strips")
    R = n // N
    if R < 2:
        raise ValueError("each strip needs at least two node lines")
    if direction in ("BT", "LR"):
        rng = [(s * R, s * R + R - 1) for s in range(N)]
        rng[-1] = (rng[-1][0], n)
        return rng
    if direction in ("TB", "RL"):
        # mirror image: the strip visited last (the first line block) owns R + 1 lines
        return [(n - (s * R + R - 1), n - s * R) if s < N - 1 else (0, R) for s in range(N)]
    raise ValueError(direction)


def orientation(direction: str) -> str:
    """'row' strips (lines j) for BT/TB, 'col' strips (lines i) for LR/RL."""
    return "row" if direction in ("BT", "TB") else "col"


def strip_matrix(k: float, n: int, a: int, b: int, orient: str, far: int = 0):
    """D_s for the strip owning lines [a, b]: returns (D (CSR, local order), global indices).

    far = +1 when the unvisited strips lie at larger line index (BT, LR), -1 when they lie at
    smaller index (TB, RL), 0 for a strip with no far neighbour (the last one visited, or
    N = 1).  The cell layer on the far side is assembled with the strip and the extra node
    line it brings is dropped; impedance is applied on every rectangle side except the far
    one."""
    lo, hi = a, b
    if far > 0:
        hi, sides_t = b + 1, "B"
    elif far < 0:
        lo, sides_t = a - 1, "T"
    else:
        sides_t = "BT"
    if orient == "row":
        K, M, MG, glob = fem.assemble_rect(n, 0, n, lo, hi, "row", sides_t + "LR")
    else:
        # column strips: lines are i; the rectangle's B/T sides are i = lo / i = hi
        sides = "".join({"B": "L", "T": "R"}[c] for c in sides_t) + "BT"
        K, M, MG, glob = fem.assemble_rect(n, lo, hi, 0, n, "col", sides)
    D = fem.helmholtz_matrix(K, M, MG, k)
    keep = np.arange((b - a + 1) * (n + 1)) + ((n + 1) if far < 0 else 0)
    return D[keep][:, keep].tocsr(), glob[keep]


def far_side(direction: str, s: int, N: int) -> int:
    """+1 / -1 for the side of the not-yet-visited strips; 0 for the last strip."""
    if s == N - 1:
        return 0
    return 1 if direction in ("BT", "LR") else -1


def to_band(D, kl: int, ku: int) -> np.ndarray:
    """LAPACK general-band storage with kl extra rows for the LU fill (zgbtrf layout)."""
    D = D.tocoo()
    nrow = D.shape[0]
    ab = np.zeros((2 * kl + ku + 1, nrow), dtype=np.complex128)
    if np.any(np.abs(D.row - D.col) > max(kl, ku)):
        raise ValueError("matrix entry outside the band")
    np.add.at(ab, (kl + ku + D.row - D.col, D.col), D.data)
    return ab


class BandLU:
    """Pivoted banded LU factorisation of one strip matrix (zgbtrf), solves by zgbtrs."""

    def __init__(self, D, bw: int):
        self.kl = self.ku = bw
        self.n = D.shape[0]
        ab = to_band(D, bw, bw)
        self.lu, self.piv, info = lapack.zgbtrf(ab, bw, bw)
        if info != 0:
            raise np.linalg.LinAlgError(f"zgbtrf info={info}")

    def solve(self, rhs: np.ndarray) -> np.ndarray:
        x, info = lapack.zgbtrs(self.lu, self.kl, self.ku, rhs.reshape(self.n, -1).astype(np.complex128),
                                self.piv)
        if info != 0:
            raise np.linalg.LinAlgError(f"zgbtrs info={info}")
        return x.reshape(rhs.shape)


class DenseLU:
    """Dense pivoted LU (tiny grids only; used when a strip block is replaced by a dense one)."""

    def __init__(self, D: np.ndarray):
        import scipy.linalg as sla
        self.n = D.shape[0]
        self.f = sla.lu_factor(D)

    def solve(self, rhs: np.ndarray) -> np.ndarray:
        import scipy.linalg as sla
        return sla.lu_solve(self.f, rhs.reshape(self.n, -1)).reshape(rhs.shape)


class FactorCache:
    """Factorisations keyed by EXACT entrywise equality of the strip matrix.

    With constant k every strip with the same line count has the same matrix, and a
    column strip in its own numbering equals the row strip of the same size, so a few
    factorisations serve every direction.  ``enabled=False`` factorises every strip."""

    def __init__(self, enabled: bool = True):
        self.enabled = enabled
        self.entries: list[tuple] = []
        self.factorisations = 0

    def get(self, D, bw: int) -> BandLU:
        if self.enabled:
            Dc = D.tocsr()
            Dc.sort_indices()
            for (shape, indptr, indices, data, lu) in self.entries:
                if (shape == Dc.shape and np.array_equal(indptr, Dc.indptr)
                        and np.array_equal(indices, Dc.indices) and np.array_equal(data, Dc.data)):
                    return lu
        lu = BandLU(D, bw)
        self.factorisations += 1
        if self.enabled:
            self.entries.append((Dc.shape, Dc.indptr.copy(), Dc.indices.copy(), Dc.data.copy(), lu))
        return lu


class Sweeper:
    """Directional double (or single) sweep preconditioner M_d^{-1} for one direction."""

    def __init__(self, A, k: float, n: int, N: int, direction: str, cache: FactorCache | None = None,
                 strip_override=None):
        self.k, self.n, self.N, self.direction = k, n, N, direction
        self.m = n + 1
        orient = orientation(direction)
        self.lines = strip_lines(n, N, direction)
        self.cache = cache if cache is not None else FactorCache()
        self.glob, self.lu = [], []
        for s, (a, b) in enumerate(self.lines):
            D, glob = strip_matrix(k, n, a, b, orient, far_side(direction, s, N))
            self.glob.append(glob)
            if strip_override is not None:
                self.lu.append(DenseLU(np.asarray(strip_override(s, D, glob))))
            else:
                self.lu.append(self.cache.get(D, self.m + 1))
        A = A.tocsr()
        # couplings of each strip to its predecessor / successor in the sweep order
        self.c_prev = [None] + [A[self.glob[s]][:, self.glob[s - 1]].tocsr() for s in range(1, N)]
        self.c_next = [A[self.glob[s]][:, self.glob[s + 1]].tocsr() for s in range(N - 1)] + [None]

    def apply(self, r: np.ndarray, double: bool = True) -> np.ndarray:
        N = self.N
        v = [None] * N
        for s in range(N):
            rhs = r[self.glob[s]].astype(np.complex128)
            if s > 0:
                rhs = rhs - self.c_prev[s] @ v[s - 1]
            v[s] = self.lu[s].solve(rhs)
        u = list(v)
        if double:
            for s in range(N - 2, -1, -1):
                u[s] = v[s] - self.lu[s].solve(self.c_next[s] @ u[s + 1])
        z = np.zeros(self.m * self.m, dtype=np.complex128)
        for s in range(N):
            z[self.glob[s]] = u[s]
        return z


def make_preconditioners(A, k: float, n: int, N: int, dirs, double: bool = True,
                         cache: FactorCache | None = None):
    """List of callables r -> M_d^{-1} r, one per direction in ``dirs`` (order kept)."""
    cache = cache if cache is not None else FactorCache()
    out = []
    for d in dirs:
        sw = Sweeper(A, k, n, N, d, cache)
        out.append(lambda r, sw=sw: sw.apply(r, double))
    return out


def block_operators(A, k: float, n: int, N: int, direction: str):
    """Dense (D + L), D, (D + U) of the block Gauss-Seidel splitting in the sweep ordering
    (tiny grids only; used to form M explicitly)."""
    sw = Sweeper(A, k, n, N, direction, FactorCache(False))
    perm = np.concatenate(sw.glob)
    Ap = A.tocsr()[perm][:, perm].toarray()
    orient = orientation(direction)
    Dblk = np.zeros_like(Ap)
    off = 0
    for s, (a, b) in enumerate(sw.lines):
        D, _ = strip_matrix(k, n, a, b, orient, far_side(direction, s, N))
        sz = D.shape[0]
        Dblk[off:off + sz, off:off + sz] = D.toarray()
        off += sz
    Lower = np.tril(Ap - np.diag(np.diag(Ap)), 0)
    Upper = np.triu(Ap - np.diag(np.diag(Ap)), 0)
    # keep only inter-strip parts of the strictly lower / upper triangles
    mask = np.zeros_like(Ap, dtype=bool)
    off = 0
    for (a, b) in sw.lines:
        sz = (b - a + 1) * (n + 1)
        mask[off:off + sz, off:off + sz] = True
        off += sz
    Lower[mask] = 0
    Upper[mask] = 0
    return perm, Dblk + Lower, Dblk, Dblk + Upper


def exact_schur_override(A, n: int, N: int, direction: str):
    """Strip override that replaces each D_s by the exact forward Schur complement
    S_s = A_ss - A_{s,prev} S_prev^{-1} A_{prev,s} (dense; tiny grids only).  With these
    blocks the double sweep is an exact block LU solve, so M = A (Section 2: an exact
    transparent condition makes the double sweep nilpotent and exact)."""
    A = A.tocsr()
    lines = strip_lines(n, N, direction)
    orient = orientation(direction)
    globs = []
    for s, (a, b) in enumerate(lines):
        _, glob = strip_matrix(1.0, n, a, b, orient, far_side(direction, s, N))
        globs.append(glob)
    S = []
    for s in range(N):
        Ass = A[globs[s]][:, globs[s]].toarray()
        if s > 0:
            Asp = A[globs[s]][:, globs[s - 1]].toarray()
            Aps = A[globs[s - 1]][:, globs[s]].toarray()
            Ass = Ass - Asp @ np.linalg.solve(S[s - 1], Aps)
        S.append(Ass)
    return lambda s, D, glob: S[s]
