"""Pins of the oracle's discretisation against facts fixed outside the oracle itself.

* closed-form stencil entries, derived by hand from the P1 right-triangle mesh;
* invariants: K 1 = 0, total mass = area, boundary mass = perimeter, A^T = A;
* a brute-force element loop written with a different formula (cross products for the
  area and edge normals for the gradients);
* O(h^2) convergence to an exact plane wave with inhomogeneous impedance data;
* the banded direct solve against numpy's dense LU.
"""
import numpy as np
import pytest

from oracle import direct, fem


def _A(k, n):
    return fem.global_system(k, n)


@pytest.mark.parametrize("k,n", [(20.0, 32), (7.5, 9)])
def test_closed_form_stencil(k, n):
    A, K, M, MG = _A(k, n)
    A = A.toarray()
    m, h = n + 1, 1.0 / n
    kh2 = (k * h) ** 2
    g = lambda i, j: j * m + i
    # interior node
    i, j = 3, 4
    c = g(i, j)
    assert A[c, c] == pytest.approx(4 - kh2 / 2, abs=1e-14)
    for nb in (g(i + 1, j), g(i - 1, j), g(i, j + 1), g(i, j - 1)):
        assert A[c, nb] == pytest.approx(-1 - kh2 / 12, abs=1e-14)
    for nb in (g(i + 1, j + 1), g(i - 1, j - 1)):
        assert A[c, nb] == pytest.approx(-kh2 / 12, abs=1e-14)
    for nb in (g(i - 1, j + 1), g(i + 1, j - 1)):
        assert A[c, nb] == 0
    assert np.count_nonzero(A[c]) == 7
    # bottom edge node
    i, j = 2, 0
    c = g(i, j)
    assert A[c, c] == pytest.approx(2 - kh2 / 4 - 1j * k * 2 * h / 3, abs=1e-14)
    for nb in (g(i + 1, 0), g(i - 1, 0)):
        assert A[c, nb] == pytest.approx(-0.5 - kh2 / 24 - 1j * k * h / 6, abs=1e-14)
    assert A[c, g(i, 1)] == pytest.approx(-1 - kh2 / 12, abs=1e-14)
    assert A[c, g(i + 1, 1)] == pytest.approx(-kh2 / 12, abs=1e-14)
    assert A[c, g(i - 1, 1)] == 0
    # corners: two triangles meet at (0,0) and (n,n), one at (n,0) and (0,n)
    for (ci, cj), kd, md in [((0, 0), 1.0, 1 / 6), ((n, n), 1.0, 1 / 6), ((n, 0), 1.0, 1 / 12),
                             ((0, n), 1.0, 1 / 12)]:
        c = g(ci, cj)
        assert A[c, c] == pytest.approx(kd - k * k * md * h * h - 1j * k * 2 * h / 3, abs=1e-14)


def test_invariants():
    A, K, M, MG = _A(13.0, 12)
    one = np.ones(K.shape[0])
    assert np.abs(K @ one).max() < 1e-13
    assert M.sum() == pytest.approx(1.0, abs=1e-13)
    assert MG.sum() == pytest.approx(4.0, abs=1e-13)
    assert abs(A - A.T).max() == 0
    # mass of a linear function: integral of x over the square = 1/2
    x, y = fem.node_coords(12)
    assert one @ (M @ x) == pytest.approx(0.5, abs=1e-13)
    # boundary integral of x over the perimeter = 0 + 1 + 1/2 + 1/2 = 2
    assert one @ (MG @ x) == pytest.approx(2.0, abs=1e-13)


def _bruteforce(k, n):
    """Independent element loop: area by cross product, gradients from edge normals."""
    m, h = n + 1, 1.0 / n
    N = m * m
    A = np.zeros((N, N), dtype=complex)
    for cj in range(n):
        for ci in range(n):
            for tri in (((ci, cj), (ci + 1, cj), (ci + 1, cj + 1)), ((ci, cj), (ci + 1, cj + 1), (ci, cj + 1))):
                P = [np.array([a * h, b * h]) for a, b in tri]
                ids = [b * m + a for a, b in tri]
                e1, e2 = P[1] - P[0], P[2] - P[0]
                area = 0.5 * abs(e1[0] * e2[1] - e1[1] * e2[0])
                grads = []
                for a in range(3):
                    e = P[(a + 2) % 3] - P[(a + 1) % 3]          # opposite edge
                    nrm = np.array([e[1], -e[0]])                  # normal to it
                    # orient towards vertex a, scale: grad = nrm / (nrm . (P_a - P_{a+1}))
                    grads.append(nrm / (nrm @ (P[a] - P[(a + 1) % 3])))
                for a in range(3):
                    for b in range(3):
                        kab = area * grads[a] @ grads[b]
                        mab = area / 6 if a == b else area / 12
                        A[ids[a], ids[b]] += kab - k * k * mab
    for side in range(4):
        for t in range(n):
            if side == 0:
                e = (t, t + 1)
            elif side == 1:
                e = (n * m + t, n * m + t + 1)
            elif side == 2:
                e = (t * m, (t + 1) * m)
            else:
                e = (t * m + n, (t + 1) * m + n)
            for a in range(2):
                for b in range(2):
                    A[e[a], e[b]] -= 1j * k * (h / 3 if a == b else h / 6)
    return A


@pytest.mark.parametrize("k,n", [(5.0, 3), (11.0, 6)])
def test_bruteforce_assembly(k, n):
    A, *_ = _A(k, n)
    assert np.abs(A.toarray() - _bruteforce(k, n)).max() < 1e-13


def test_plane_wave_second_order():
    """Nodal error to u = exp(i k d.x) with impedance data g = i k (d.nu - 1) u decays as
    O(h^2) (P1 elements, smooth solution)."""
    k = 10.0
    errs, hs = [], []
    for n in (32, 64, 128, 256):
        A, *_ = _A(k, n)
        u, b = fem.plane_wave(k, n)
        x = direct.solve(A, b, n)
        errs.append(np.linalg.norm(x - u) / np.linalg.norm(u))
        hs.append(1.0 / n)
    rates = np.diff(np.log(errs)) / np.diff(np.log(hs))
    assert errs[-1] < 2e-3
    assert np.all(rates > 1.8) and np.all(rates < 2.2), (errs, rates)


@pytest.mark.parametrize("n", [4, 8, 16])
def test_banded_direct_vs_dense(n):
    k = 9.0
    A, K, M, MG = _A(k, n)
    rng = np.random.default_rng(1)
    b = rng.standard_normal(A.shape[0]) + 1j * rng.standard_normal(A.shape[0])
    x = direct.solve(A, b, n)
    xd = direct.dense_solve(A, b)
    assert np.linalg.norm(x - xd) / np.linalg.norm(xd) < 1e-12
    assert np.linalg.norm(A @ x - b) / np.linalg.norm(b) < 1e-12


def test_load_vector_constant_source():
    """f = 1 everywhere: b = -M 1, whose entries sum to -area."""
    n = 10
    _, M, MG, _ = fem.assemble_rect(n, 0, n, 0, n)
    b = fem.load_vector(n, M, MG, np.ones((n + 1) ** 2))
    assert b.sum() == pytest.approx(-1.0, abs=1e-13)
    # Gaussian far narrower than the domain: integral ~ 2 pi sigma^2 amp
    n = 256
    _, M, MG, _ = fem.assemble_rect(n, 0, n, 0, n)
    src = np.array([[0.5, 0.5, 0.05, 2.0, -1.0]])
    b = fem.load_vector(n, M, MG, fem.gaussian_source(n, src))
    assert b.sum() == pytest.approx(-(2 - 1j) * 2 * np.pi * 0.05 ** 2, rel=1e-4)
