"""P1 finite elements for  Delta u + k^2 u = f  in (0,1)^2,  du/dn - i k u = g  on the boundary.

Problem statement: Section 1, Eq. (1a)-(1b).  Weak form (test function v, no complex
conjugation, integrate Delta u v by parts and substitute du/dn = g + i k u):

    int grad u . grad v  -  k^2 int u v  -  i k int_Gamma u v  =  - int f v  +  int_Gamma g v

so  A = K - k^2 M - i k M_Gamma  and  b = -M f_I + M_Gamma g_I  with nodal interpolants
f_I, g_I.  A is complex symmetric (A^T = A), not Hermitian.

Mesh: nodes (i, j), x = i h, y = j h, 0 <= i, j <= n, global index g = j * (n + 1) + i.
Every cell [i, i+1] x [j, j+1] is cut along its SW-NE diagonal into
    T1 = {(i, j), (i+1, j), (i+1, j+1)}   and   T2 = {(i, j), (i+1, j+1), (i, j+1)}.
Element matrices are computed from the barycentric gradients of each triangle.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp

# vertex offsets (di, dj) of the two triangle types of a cell
T1 = ((0, 0), (1, 0), (1, 1))
T2 = ((0, 0), (1, 1), (0, 1))


def element_matrices(h: float, tri) -> tuple[np.ndarray, np.ndarray]:
    """Local P1 stiffness and consistent mass matrices of one triangle (vertex offsets tri)."""
    p = np.array(tri, dtype=np.float64) * h
    e1, e2 = p[1] - p[0], p[2] - p[0]
    det = e1[0] * e2[1] - e1[1] * e2[0]
    area = 0.5 * abs(det)
    # gradients of the barycentric coordinates: solve J^T grad(lambda_{1,2}) = e_{1,2}
    J = np.array([e1, e2]).T
    G12 = np.linalg.solve(J.T, np.eye(2))          # columns = grad lambda_1, grad lambda_2
    g1, g2 = G12[:, 0], G12[:, 1]
    g0 = -(g1 + g2)
    grads = np.array([g0, g1, g2])
    Kloc = area * grads @ grads.T
    Mloc = (area / 12.0) * (np.ones((3, 3)) + np.eye(3))
    return Kloc, Mloc


def edge_mass(length: float) -> np.ndarray:
    """Consistent P1 mass matrix of one boundary edge."""
    return (length / 6.0) * np.array([[2.0, 1.0], [1.0, 2.0]])


def assemble_rect(n: int, i0: int, i1: int, j0: int, j1: int, order: str = "row",
                  sides: str = "BTLR"):
    """K, M, M_Gamma of the P1 problem posed on the node rectangle [i0, i1] x [j0, j1].

    Only cells inside the rectangle contribute; M_Gamma is taken over the rectangle sides
    named in ``sides`` (B: j = j0, T: j = j1, L: i = i0, R: i = i1).  Local numbering:
    order='row' -> (j - j0) * ni + (i - i0); order='col' -> (i - i0) * nj + (j - j0).
    Returns CSR matrices and the global node indices (g = j * (n + 1) + i) in local order.
    """
    h = 1.0 / n
    m = n + 1
    ni, nj = i1 - i0 + 1, j1 - j0 + 1

    def lidx(i, j):
        if order == "row":
            return (j - j0) * ni + (i - i0)
        return (i - i0) * nj + (j - j0)

    nloc = ni * nj
    rows, cols, kv, mv = [], [], [], []
    ci, cj = np.meshgrid(np.arange(i0, i1), np.arange(j0, j1), indexing="ij")
    ci, cj = ci.ravel(), cj.ravel()
    for tri in (T1, T2):
        Kloc, Mloc = element_matrices(h, tri)
        vid = [lidx(ci + di, cj + dj) for (di, dj) in tri]
        for a in range(3):
            for b in range(3):
                rows.append(vid[a])
                cols.append(vid[b])
                kv.append(np.full(ci.size, Kloc[a, b]))
                mv.append(np.full(ci.size, Mloc[a, b]))
    rows = np.concatenate(rows) if rows else np.zeros(0, int)
    cols = np.concatenate(cols) if cols else np.zeros(0, int)
    K = sp.coo_matrix((np.concatenate(kv), (rows, cols)), shape=(nloc, nloc)).tocsr()
    M = sp.coo_matrix((np.concatenate(mv), (rows, cols)), shape=(nloc, nloc)).tocsr()

    # boundary edges of the rectangle, each of length h
    Eloc = edge_mass(h)
    ea, eb = [np.zeros(0, dtype=np.int64)], [np.zeros(0, dtype=np.int64)]
    xs = np.arange(i0, i1)
    ys = np.arange(j0, j1)
    if "B" in sides:
        ea.append(lidx(xs, np.full_like(xs, j0)))
        eb.append(lidx(xs + 1, np.full_like(xs, j0)))
    if "T" in sides:
        ea.append(lidx(xs, np.full_like(xs, j1)))
        eb.append(lidx(xs + 1, np.full_like(xs, j1)))
    if "L" in sides:
        ea.append(lidx(np.full_like(ys, i0), ys))
        eb.append(lidx(np.full_like(ys, i0), ys + 1))
    if "R" in sides:
        ea.append(lidx(np.full_like(ys, i1), ys))
        eb.append(lidx(np.full_like(ys, i1), ys + 1))
    ea, eb = np.concatenate(ea), np.concatenate(eb)
    gr = np.concatenate([ea, ea, eb, eb])
    gc = np.concatenate([ea, eb, ea, eb])
    gv = np.concatenate([np.full(ea.size, Eloc[0, 0]), np.full(ea.size, Eloc[0, 1]),
                         np.full(ea.size, Eloc[1, 0]), np.full(ea.size, Eloc[1, 1])])
    MG = sp.coo_matrix((gv, (gr, gc)), shape=(nloc, nloc)).tocsr()

    II, JJ = np.meshgrid(np.arange(i0, i1 + 1), np.arange(j0, j1 + 1), indexing="ij")
    glob = np.empty(nloc, dtype=np.int64)
    glob[lidx(II.ravel(), JJ.ravel())] = JJ.ravel() * m + II.ravel()
    return K, M, MG, glob


def helmholtz_matrix(K, M, MG, k: float):
    """A = K - k^2 M - i k M_Gamma (complex128 CSR)."""
    return (K.astype(np.complex128) - (k * k) * M - 1j * k * MG).tocsr()


def global_system(k: float, n: int):
    """Global matrices on the unit square: returns (A, K, M, MG)."""
    K, M, MG, _ = assemble_rect(n, 0, n, 0, n, "row")
    return helmholtz_matrix(K, M, MG, k), K, M, MG


def node_coords(n: int) -> tuple[np.ndarray, np.ndarray]:
    """x, y of every node in global order g = j * (n + 1) + i."""
    t = np.arange(n + 1) / n
    X, Y = np.meshgrid(t, t, indexing="xy")
    return X.ravel(), Y.ravel()


def gaussian_source(n: int, sources: np.ndarray) -> np.ndarray:
    """Nodal values f_I of a sum of Gaussians, rows (x0, y0, sigma, re, im)."""
    x, y = node_coords(n)
    f = np.zeros(x.size, dtype=np.complex128)
    for x0, y0, sig, re, im in np.atleast_2d(sources):
        f += (re + 1j * im) * np.exp(-((x - x0) ** 2 + (y - y0) ** 2) / (2.0 * sig * sig))
    return f


def load_vector(n: int, M, MG, f_nodal: np.ndarray, g_nodal: np.ndarray | None = None) -> np.ndarray:
    """b = -M f_I + M_Gamma g_I."""
    b = -(M @ f_nodal.astype(np.complex128))
    if g_nodal is not None:
        b = b + MG @ g_nodal.astype(np.complex128)
    return b


def gaussian_rhs(k: float, n: int, sources: np.ndarray) -> np.ndarray:
    """Load vector of the impedance problem with a Gaussian source and g = 0."""
    _, M, _, _ = assemble_rect(n, 0, n, 0, n, "row")
    return load_vector(n, M, None, gaussian_source(n, sources))


def plane_wave(k: float, n: int, theta: float = 0.3):
    """Exact plane wave u = exp(i k d.x), d = (cos theta, sin theta), with f = 0 and the
    impedance data g = du/dn - i k u = i k (d.nu - 1) u on each side (corners: the
    consistent boundary mass pairs each boundary edge with its own outward normal).
    Returns (u_exact nodal, b)."""
    d = np.array([np.cos(theta), np.sin(theta)])
    x, y = node_coords(n)
    u = np.exp(1j * k * (d[0] * x + d[1] * y))
    h = 1.0 / n
    m = n + 1
    b = np.zeros(m * m, dtype=np.complex128)
    Eloc = edge_mass(h)
    # integrate g v over each boundary edge with the edge's own normal (exact-in-g_I sense)
    for normal, edges in _boundary_edges(n):
        gn = 1j * k * (d @ np.array(normal) - 1.0) * u
        for ga, gb in edges:
            b[ga] += Eloc[0, 0] * gn[ga] + Eloc[0, 1] * gn[gb]
            b[gb] += Eloc[1, 0] * gn[ga] + Eloc[1, 1] * gn[gb]
    return u, b


def _boundary_edges(n: int):
    m = n + 1
    ii = np.arange(n)
    bottom = [(i, i + 1) for i in ii]
    top = [(n * m + i, n * m + i + 1) for i in ii]
    left = [(j * m, (j + 1) * m) for j in ii]
    right = [(j * m + n, (j + 1) * m + n) for j in ii]
    return [((0.0, -1.0), bottom), ((0.0, 1.0), top), ((-1.0, 0.0), left), ((1.0, 0.0), right)]
