"""The paper's own discretisation and decomposition (Section 4), as a second mode of the oracle:
five-point finite differences and overlapping strips whose sweeps pass Robin data (Section 2,
Eqs. (2)-(4)), where a node shared by two subdomains keeps whichever of their solutions was
computed last.

Test infrastructure only, like the rest of oracle/: plain numpy/scipy, FP64.

Discretisation (Section 4): five-point finite differences on a uniform square grid.  Nodes (i, j) at (i h, j h), 0 <= i, j <= n, h = 1/n, index
g = j (n+1) + i.  The row of an interior node is Eq. (1a) times -h^2:
    (4 - k^2 h^2) u - (sum of the four neighbours) = -h^2 f.
Reading (the paper does not say how the Robin condition Eq. (1b) enters the scheme): a ghost
node beyond each boundary side, du/dn by the centred difference (u_ghost - u_inward) / (2h),
and the ghost eliminated with du/dn - i k u = g; edge rows are halved and corner rows quartered,
which makes the matrix complex symmetric:
    edge:    (2 - k^2 h^2/2 - i k h) u - u_inward - (u_along1 + u_along2)/2 = -h^2 f/2 + h g
    corner:  (1 - k^2 h^2/4 - i k h) u - (u_inward1 + u_inward2)/2 = -h^2 f/4 + h (g1 + g2)/2
(g = 0 on the physical boundary).  Row scale s = 1, 1/2, 1/4 (interior, edge, corner).

Decomposition (Section 4): the cells are split into N strips of R = n/N cell layers across the
sweep direction, strip s between node lines sR and (s+1)R, and every strip is extended by one
line of nodes across each internal boundary: subdomain s owns node lines
max(0, sR - 1) .. min(n, (s+1)R + 1), so that neighbours overlap by 2h (three node lines).
Subdomain problems are the same five-point Robin problem on the subdomain's rectangle (the
transmission operator of Eq. (4) is the boundary condition of Eq. (1b)): the matrix of the
rectangle with ghost-node Robin rows on all four sides.  The right-hand side of a subdomain for
a residual r is (s_sub / s_glob) r on its nodes (the global rows rescaled to the subdomain's
row scales) plus s_sub 2 h g on its artificial boundary rows, where g is the Robin data
B(w) = dw/dn - i k w of the neighbour's solution w at that line, by the same centred
difference (Eqs. (2b), (3b), (3c)).

Double sweep (Eqs. (2)-(3)): forward v_s with data B(v_{s-1}) on Gamma_{s,1} and 0 on
Gamma_{s,2}; backward u_s with data B(v_{s-1}) on Gamma_{s,1} and B(u_{s+1}) on Gamma_{s,2},
u_N = v_N.  Output (Section 2, end): every node takes the value of the most recent subdomain
solve that contains it -- after a double sweep the lower subdomain of an overlap (u_s is solved
after u_{s+1}), after a forward sweep the higher one.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp

from . import mpgmres, sweep

DIRECTIONS = ("LR", "RL", "BT", "TB")


def _row_scale(i, j, i0, i1, j0, j1):
    return (0.5 if i in (i0, i1) else 1.0) * (0.5 if j in (j0, j1) else 1.0)


def rect_matrix(k: float, n: int, i0: int, i1: int, j0: int, j1: int) -> sp.csr_matrix:
    """Five-point Robin matrix of the node rectangle [i0, i1] x [j0, j1] (ghost-node Robin rows
    on all four sides), local numbering (j - j0) (i1 - i0 + 1) + (i - i0).

    Unscaled row of node p: centre 4 - k^2 h^2, -1 per neighbour; a side of p on the
    rectangle's boundary has a ghost node instead of a neighbour, which the Robin condition
    replaces by the mirror (inward) neighbour, so that neighbour's coefficient doubles to -2,
    and adds -2 i k h to the centre.  The row is then multiplied by its scale s (1/2 per
    boundary side)."""
    h = 1.0 / n
    kh2, ikh = (k * h) ** 2, 1j * k * h
    ni, nj = i1 - i0 + 1, j1 - j0 + 1
    I, J = np.meshgrid(np.arange(ni), np.arange(nj))
    I, J = I.ravel(), J.ravel()
    g = J * ni + I
    s = np.where((I == 0) | (I == ni - 1), 0.5, 1.0) * np.where((J == 0) | (J == nj - 1), 0.5, 1.0)
    nsides = ((I == 0).astype(int) + (I == ni - 1) + (J == 0) + (J == nj - 1))
    rows, cols, vals = [g], [g], [s * (4.0 - kh2 - 2.0 * ikh * nsides)]
    for di, dj in ((1, 0), (-1, 0), (0, 1), (0, -1)):
        ii, jj = I + di, J + dj
        inside = (ii >= 0) & (ii < ni) & (jj >= 0) & (jj < nj)
        # outside: the ghost, replaced by the mirror node (which is inside for n >= 1)
        ti = np.where(inside, ii, I - di)
        tj = np.where(inside, jj, J - dj)
        rows.append(g)
        cols.append(tj * ni + ti)
        vals.append(-s)
    return sp.csr_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                         shape=(ni * nj, ni * nj)).astype(np.complex128)


def global_matrix(k: float, n: int) -> sp.csr_matrix:
    return rect_matrix(k, n, 0, n, 0, n)


def row_scales(n: int, i0: int, i1: int, j0: int, j1: int) -> np.ndarray:
    out = np.empty((j1 - j0 + 1) * (i1 - i0 + 1))
    q = 0
    for j in range(j0, j1 + 1):
        for i in range(i0, i1 + 1):
            out[q] = _row_scale(i, j, i0, i1, j0, j1)
            q += 1
    return out


def load_vector(n: int, f_nodal: np.ndarray, g_sides=None) -> np.ndarray:
    """b = s (-h^2 f) + s 2 h (sum of the Robin data g of the node's boundary sides); g_sides:
    dict side -> nodal array (sides 'L', 'R', 'B', 'T'), None for g = 0."""
    h = 1.0 / n
    m = n + 1
    s = row_scales(n, 0, n, 0, n)
    b = s * (-h * h) * np.asarray(f_nodal, dtype=np.complex128)
    if g_sides:
        I, J = np.meshgrid(np.arange(m), np.arange(m))
        I, J = I.ravel(), J.ravel()
        on = {"L": I == 0, "R": I == n, "B": J == 0, "T": J == n}
        for side, g in g_sides.items():
            b = b + np.where(on[side], s * 2.0 * h * np.asarray(g), 0.0)
    return b


def paper_source(k: float, n: int) -> np.ndarray:
    """Section 4's benchmark source f = 3e4 exp(-200 k ((x - 0.5)^2 + (y - 0.5)^2)), nodal."""
    x = np.arange(n + 1) / n
    X, Y = np.meshgrid(x, x)
    return (3e4 * np.exp(-200.0 * k * ((X - 0.5) ** 2 + (Y - 0.5) ** 2))).ravel().astype(np.complex128)


def frame_perm(n: int, direction: str) -> np.ndarray:
    """perm[q] = global index of frame node q = l (n+1) + i, where l counts the node lines in the
    sweep direction (BT: j, TB: n - j, LR: i, RL: n - i) and i runs along the line."""
    m = n + 1
    L, I = np.meshgrid(np.arange(m), np.arange(m), indexing="ij")
    if direction == "BT":
        gi, gj = I, L
    elif direction == "TB":
        gi, gj = I, n - L
    elif direction == "LR":
        gi, gj = L, I
    elif direction == "RL":
        gi, gj = n - L, I
    else:
        raise ValueError(direction)
    return (gj * m + gi).ravel()


class OverlapSweeper:
    """Double (or forward) sweep of Section 2 over overlapping strips for one direction, in the
    direction's frame (the five-point Robin problem is invariant under the square's symmetries,
    so every direction is a bottom-to-top sweep of a relabelled vector)."""

    def __init__(self, k: float, n: int, N: int, direction: str):
        if n % N:
            raise ValueError("n must be a multiple of the number of strips")
        self.k, self.n, self.N, self.m = k, n, N, n + 1
        self.h = 1.0 / n
        R = n // N
        self.perm = frame_perm(n, direction)
        self.lines = [(max(0, s * R - 1), min(n, (s + 1) * R + 1)) for s in range(N)]
        cache = {}
        self.lu = []
        for (a, b) in self.lines:
            key = (b - a, a == 0, b == n)
            if key not in cache:
                cache[key] = sweep.BandLU(rect_matrix(k, n, 0, n, a, b), self.m + 1)
            self.lu.append(cache[key])
        self.s_glob = row_scales(n, 0, n, 0, n).reshape(self.m, self.m)
        self.s_sub = [row_scales(n, 0, n, a, b).reshape(b - a + 1, self.m) for (a, b) in self.lines]

    def _data(self, w_lines: np.ndarray, a_w: int, p: int, outward: int) -> np.ndarray:
        """Robin data B(w) = dw/dn - i k w on frame line p of w (which holds lines a_w..),
        outward = -1 (normal towards lower lines) or +1."""
        wp = w_lines[p - a_w]
        dn = (w_lines[p + outward - a_w] - w_lines[p - outward - a_w]) / (2.0 * self.h)
        return dn - 1j * self.k * wp

    def _solve(self, s: int, rf: np.ndarray, g_lo=None, g_hi=None) -> np.ndarray:
        a, b = self.lines[s]
        rhs = (self.s_sub[s] / self.s_glob[a:b + 1]) * rf[a:b + 1]
        if g_lo is not None:
            rhs[0] = rhs[0] + self.s_sub[s][0] * 2.0 * self.h * g_lo
        if g_hi is not None:
            rhs[-1] = rhs[-1] + self.s_sub[s][-1] * 2.0 * self.h * g_hi
        return self.lu[s].solve(rhs.ravel()).reshape(b - a + 1, self.m)

    def apply(self, r: np.ndarray, double: bool = True, parts: list | None = None) -> np.ndarray:
        """M_d^{-1} r; if `parts` is a list, the subdomain solutions (frame lines a..b of each,
        the last computed one per subdomain) are appended to it."""
        N = self.N
        rf = np.asarray(r, dtype=np.complex128)[self.perm].reshape(self.m, self.m)
        v = [None] * N
        for s in range(N):
            g_lo = None
            if s > 0:
                a, _ = self.lines[s]
                g_lo = self._data(v[s - 1], self.lines[s - 1][0], a, -1)
            v[s] = self._solve(s, rf, g_lo, None)
        z = np.zeros((self.m, self.m), dtype=np.complex128)
        if not double:
            for s in range(N):  # increasing s: overlaps keep the later (higher) strip's values
                a, b = self.lines[s]
                z[a:b + 1] = v[s]
            if parts is not None:
                parts.extend(v)
        else:
            u = [None] * N
            u[N - 1] = v[N - 1]
            for s in range(N - 2, -1, -1):
                g_lo = None
                if s > 0:
                    g_lo = self._data(v[s - 1], self.lines[s - 1][0], self.lines[s][0], -1)
                g_hi = self._data(u[s + 1], self.lines[s + 1][0], self.lines[s][1], +1)
                u[s] = self._solve(s, rf, g_lo, g_hi)
            for s in range(N - 1, -1, -1):  # decreasing s: overlaps keep the lower strip's values
                a, b = self.lines[s]
                z[a:b + 1] = u[s]
            if parts is not None:
                parts.extend(u)
        out = np.empty(self.m * self.m, dtype=np.complex128)
        out[self.perm] = z.ravel()
        return out


class FDProblem:
    """Assembled five-point operator and the t overlapping-sweep preconditioners."""

    def __init__(self, k: float, n: int, N: int, dirs: str = "LR+BT", double: bool = True):
        self.k, self.n, self.N = k, n, N
        self.dirs = [d.strip().upper() for d in dirs.split("+") if d.strip()]
        self.A = global_matrix(k, n)
        self.sweepers = [OverlapSweeper(k, n, N, d) for d in self.dirs]
        self.double = double
        self.precs = [(lambda r, sw=sw: sw.apply(r, double)) for sw in self.sweepers]

    def paper_rhs(self) -> np.ndarray:
        return load_vector(self.n, paper_source(self.k, self.n))

    def solve(self, b: np.ndarray, tol: float, maxit: int = 200, **kw) -> mpgmres.Result:
        return mpgmres.solve(self.A, self.precs, b, tol=tol, maxit=maxit, **kw)
