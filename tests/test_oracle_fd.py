"""Pins of the oracle's second mode: the paper's five-point finite differences and overlapping
strip sweeps with Robin transmission (Section 4; Section 2, Eqs. (2)-(4)).

* the matrix entries against their closed forms (interior, edge, corner rows) and against a
  node-by-node assembly written out separately; complex symmetry;
* second-order convergence to an exact plane wave with inhomogeneous Robin data;
* a subdomain solve whose Robin data come from the exact discrete solution returns that
  solution on the subdomain (the transmission data and the row rescaling are consistent with
  the global equations);
* one strip: the sweep is the exact inverse, MPGMRES converges in one iteration;
* the four directions are relabellings of one sweep; the overlaps hold the most recent solve;
* Table 1's observation that LRL+BTB needs about half the iterations of LRL.
Parity with the paper's printed iteration counts stays unpinned: its Robin discretisation and
MATLAB's solvers are not specified beyond the text.
"""
import numpy as np
import pytest
from scipy.sparse.linalg import spsolve

from oracle import fd


def node_by_node(k, n, i0, i1, j0, j1):
    """Dense matrix of the Robin rectangle, one row at a time from the ghost-node elimination."""
    h = 1.0 / n
    ni, nj = i1 - i0 + 1, j1 - j0 + 1
    M = np.zeros((ni * nj, ni * nj), complex)
    for j in range(j0, j1 + 1):
        for i in range(i0, i1 + 1):
            row = (j - j0) * ni + (i - i0)
            centre = 4.0 - (k * h) ** 2
            coef = {}
            for di, dj in ((1, 0), (-1, 0), (0, 1), (0, -1)):
                p = (i + di, j + dj)
                if not (i0 <= p[0] <= i1 and j0 <= p[1] <= j1):
                    # ghost: u_ghost = u_mirror + 2 h (i k u + g)
                    centre -= 2j * k * h
                    p = (i - di, j - dj)
                coef[p] = coef.get(p, 0.0) - 1.0
            scale = (0.5 if i in (i0, i1) else 1.0) * (0.5 if j in (j0, j1) else 1.0)
            M[row, row] += scale * centre
            for (pi, pj), c in coef.items():
                M[row, (pj - j0) * ni + (pi - i0)] += scale * c
    return M


def test_closed_form_rows_and_symmetry():
    k, n = 7.0, 10
    h = 1.0 / n
    A = fd.global_matrix(k, n).toarray()
    m = n + 1
    g = lambda i, j: j * m + i
    assert np.allclose(A, A.T, atol=0)
    # interior
    assert A[g(4, 5), g(4, 5)] == pytest.approx(4 - (k * h) ** 2)
    for p in (g(3, 5), g(5, 5), g(4, 4), g(4, 6)):
        assert A[g(4, 5), p] == -1
    # edge (i = 0)
    assert A[g(0, 5), g(0, 5)] == pytest.approx(2 - (k * h) ** 2 / 2 - 1j * k * h)
    assert A[g(0, 5), g(1, 5)] == -1
    assert A[g(0, 5), g(0, 4)] == -0.5 and A[g(0, 5), g(0, 6)] == -0.5
    # corner
    assert A[g(0, 0), g(0, 0)] == pytest.approx(1 - (k * h) ** 2 / 4 - 1j * k * h)
    assert A[g(0, 0), g(1, 0)] == -0.5 and A[g(0, 0), g(0, 1)] == -0.5
    assert np.count_nonzero(A[g(0, 0)]) == 3


@pytest.mark.parametrize("rect", [(0, 12, 0, 12), (0, 10, 3, 7), (2, 6, 0, 9)])
def test_matrix_equals_node_by_node_assembly(rect):
    k, n = 9.0, 12
    assert np.abs(fd.rect_matrix(k, n, *rect).toarray() - node_by_node(k, n, *rect)).max() == 0


def test_plane_wave_second_order():
    k, th = 10.0, 0.3
    dx, dy = np.cos(th), np.sin(th)
    errs = []
    for n in (16, 32, 64):
        x = np.arange(n + 1) / n
        X, Y = np.meshgrid(x, x)
        ue = np.exp(1j * k * (dx * X + dy * Y)).ravel()
        # Robin data du/dn - i k u of the plane wave on each side (outward normals)
        g = {"L": 1j * k * (-dx - 1) * ue, "R": 1j * k * (dx - 1) * ue,
             "B": 1j * k * (-dy - 1) * ue, "T": 1j * k * (dy - 1) * ue}
        b = fd.load_vector(n, np.zeros((n + 1) ** 2), g)
        uh = spsolve(fd.global_matrix(k, n).tocsc(), b)
        errs.append(np.linalg.norm(uh - ue) / np.linalg.norm(ue))
    rates = np.log2(np.array(errs[:-1]) / np.array(errs[1:]))
    assert np.all((rates > 1.8) & (rates < 2.2)), (errs, rates)


@pytest.mark.parametrize("d", fd.DIRECTIONS)
def test_exact_data_reproduce_the_solution(d):
    k, n, N = 10.0, 24, 3
    A = fd.global_matrix(k, n)
    rng = np.random.default_rng(0)
    b = rng.standard_normal((n + 1) ** 2) + 1j * rng.standard_normal((n + 1) ** 2)
    u = spsolve(A.tocsc(), b)
    sw = fd.OverlapSweeper(k, n, N, d)
    bf = b[sw.perm].reshape(n + 1, n + 1)
    uf = u[sw.perm].reshape(n + 1, n + 1)
    for s in range(N):
        a, e = sw.lines[s]
        g_lo = sw._data(uf, 0, a, -1) if a > 0 else None
        g_hi = sw._data(uf, 0, e, +1) if e < n else None
        v = sw._solve(s, bf, g_lo, g_hi)
        assert np.abs(v - uf[a:e + 1]).max() < 1e-12 * np.abs(uf).max(), s


def test_one_strip_is_exact():
    k, n = 12.0, 20
    P = fd.FDProblem(k, n, 1, "LR")
    b = P.paper_rhs()
    r = P.solve(b, tol=1e-10)
    assert r.iterations == 1 and r.rel_res_explicit < 1e-12


def test_directions_are_relabellings():
    k, n, N = 8.0, 16, 4
    rng = np.random.default_rng(1)
    r = rng.standard_normal((n + 1) ** 2) + 1j * rng.standard_normal((n + 1) ** 2)
    m = n + 1
    T = np.arange(m * m).reshape(m, m).T.ravel()  # transpose: node (i, j) <-> (j, i)
    z_bt = fd.OverlapSweeper(k, n, N, "BT").apply(r[T])[T]
    z_lr = fd.OverlapSweeper(k, n, N, "LR").apply(r)
    assert np.abs(z_bt - z_lr).max() < 1e-13 * np.abs(z_lr).max()


def test_overlaps_hold_the_most_recent_solve():
    k, n, N = 8.0, 16, 4
    R = n // N
    rng = np.random.default_rng(2)
    r = rng.standard_normal((n + 1) ** 2) + 1j * rng.standard_normal((n + 1) ** 2)
    sw = fd.OverlapSweeper(k, n, N, "BT")
    for double in (True, False):
        parts = []
        z = sw.apply(r, double, parts).reshape(n + 1, n + 1)
        for s in range(N - 1):
            # node lines sR + R - 1 .. sR + R + 1 are shared by subdomains s and s + 1
            a0, a1 = sw.lines[s][0], sw.lines[s + 1][0]
            for line in range((s + 1) * R - 1, (s + 1) * R + 2):
                owner, a = (s, a0) if double else (s + 1, a1)
                assert np.array_equal(z[line], parts[owner][line - a]), (double, s, line)


def test_lrl_btb_about_halves_the_iterations():
    """k = 40, h = 1/192, 8 strips: 16 iterations with LRL, 7 with LRL+BTB."""
    k, n, N = 40.0, 192, 8
    it = {}
    try:  # the sweeps are many small sparse solves: BLAS threads only add contention
        from threadpoolctl import threadpool_limits
        limit = threadpool_limits(1)
    except ImportError:
        limit = None
    try:
        for dirs in ("LR", "LR+BT"):
            P = fd.FDProblem(k, n, N, dirs)
            it[dirs] = P.solve(P.paper_rhs(), tol=1e-6).iterations
    finally:
        if limit is not None:
            limit.unregister()
    assert it["LR+BT"] <= 0.6 * it["LR"], it
