"""Pins of the oracle's selective flexible MPGMRES (Section 3).

* one preconditioner: the residual history equals a brute-force least-squares solve over
  the explicit right-preconditioned Krylov basis (MPGMRES reduces to GMRES, Section 3);
* iteration one minimises over span{M_i^{-1} b}; iteration two over the selective space
  built by the "other preconditioner" rule of Section 4, both by brute force;
* the inner-product count of a single Gram-Schmidt pass is (k - 1/2) t^2 + (3/2) t
  (Section 3);
* Arnoldi relation A Z = V H, orthonormal V, monotone residuals;
* duplicated preconditioners deflate and reproduce the t = 1 iterates; a direction that
  agrees with another to 1e-11 of its size is deflated even when Gram-Schmidt against the
  basis has already removed most of it, and the explicit residual follows the implicit one;
* the converged solution agrees with the banded direct solve.
"""
import numpy as np
import pytest

from oracle import direct, fem, mpgmres, solver, sweep


def _setup(k=12.0, n=8, N=2, dirs="LR+RL+BT+TB"):
    P = solver.Problem(k, n, N, dirs)
    b = P.rhs(np.array([[0.45, 0.55, 0.08, 1.0, 0.5]]))
    return P, b


def _lstsq_res(A, Zcols, b):
    Z = np.array(Zcols).T
    y, *_ = np.linalg.lstsq(A @ Z, b, rcond=None)
    return np.linalg.norm(b - A @ (Z @ y)) / np.linalg.norm(b)


def test_t1_is_gmres():
    P, b = _setup(dirs="BT")
    A, Minv = P.A, P.precs[0]
    res = P.solve(b, tol=1e-14, maxit=5)
    basis = [Minv(b)]
    for it in range(5):
        expect = _lstsq_res(A, basis, b)
        assert res.history[it] == pytest.approx(expect, rel=1e-6, abs=1e-14)
        basis.append(Minv(A @ basis[-1]))


def test_first_iteration_span():
    P, b = _setup()
    res = P.solve(b, tol=1e-14, maxit=1)
    expect = _lstsq_res(P.A, [p(b) for p in P.precs], b)
    assert res.history[0] == pytest.approx(expect, rel=1e-9)


def test_second_iteration_cross_space():
    """t = 2: iteration 2 adds M_1^{-1} v2 and M_2^{-1} v1, where v_i is the new orthonormal
    vector obtained from A M_i^{-1} b (Gram-Schmidt in preconditioner order, positive
    diagonal)."""
    P, b = _setup(dirs="LR+BT")
    A = P.A
    z1, z2 = [p(b) for p in P.precs]
    Q, R = np.linalg.qr(np.array([b, A @ z1, A @ z2]).T)
    Q = Q * np.sign(np.diag(R)).conj()       # positive diagonal
    v1, v2 = Q[:, 1], Q[:, 2]
    space = [z1, z2, P.precs[0](v2), P.precs[1](v1)]
    res = P.solve(b, tol=1e-14, maxit=2)
    assert res.history[1] == pytest.approx(_lstsq_res(A, space, b), rel=1e-7)


def test_second_iteration_sum_space():
    """t > 2: iteration 2 applies every preconditioner to the sum of the new vectors."""
    P, b = _setup()
    A = P.A
    Z1 = [p(b) for p in P.precs]
    Q, R = np.linalg.qr(np.array([b] + [A @ z for z in Z1]).T)
    Q = Q * np.sign(np.diag(R)).conj()
    s = Q[:, 1:].sum(axis=1)
    space = Z1 + [p(s) for p in P.precs]
    res = P.solve(b, tol=1e-14, maxit=2)
    assert res.history[1] == pytest.approx(_lstsq_res(A, space, b), rel=1e-7)


@pytest.mark.parametrize("t", [1, 2, 3, 4])
def test_inner_product_count(t):
    P, b = _setup(dirs="+".join(sweep.DIRECTIONS[:t]), n=12, N=3)
    res = P.solve(b, tol=1e-14, maxit=4, single_pass=True)
    for k, c in enumerate(res.inner_products, start=1):
        assert c == (k - 0.5) * t * t + 1.5 * t


def test_arnoldi_relation_and_orthonormality():
    P, b = _setup(n=16, N=4)
    res = P.solve(b, tol=1e-14, maxit=6, keep_basis=True)
    V, Z, H = res.V, res.Z, res.H
    assert np.abs(V.conj().T @ V - np.eye(V.shape[1])).max() < 1e-12
    AZ = P.A @ Z
    assert np.linalg.norm(AZ - V @ H) <= 1e-12 * np.linalg.norm(AZ)
    # scalar upper Hessenberg
    assert np.all(np.abs(np.tril(H, -2)) == 0)
    assert np.all(np.diff(res.history) <= 1e-15)


def test_duplicate_preconditioners_deflate_to_t1():
    P, b = _setup(n=16, N=4, dirs="BT")
    one = P.solve(b, tol=1e-10, maxit=50)
    two = mpgmres.solve(P.A, [P.precs[0], P.precs[0]], b, tol=1e-10, maxit=50)
    assert two.iterations == one.iterations
    np.testing.assert_allclose(two.history, one.history, rtol=1e-6)
    assert np.linalg.norm(two.x - one.x) / np.linalg.norm(one.x) < 1e-9


def test_nearly_dependent_direction_is_deflated():
    """Two preconditioners of the form A^{-1}(I + 1e-3 E1), the second perturbed by 1e-11: the
    new columns A z_1, A z_2 agree to 1e-11 of their size, while projecting them on the
    basis (b) leaves only 1e-3 of it.  Measured against ||A z_j|| (the deflation reading) the
    second column is dependent and is dropped; kept (measured against the 1e-3 remainder it
    would pass a 1e-10 test), it makes the rotated triangular factor ill-conditioned and the
    explicit residual of x = Z y stalls near 1e-9 while the implicit one reaches 1e-14."""
    A, *_ = fem.global_system(10.0, 16)
    Ad = A.toarray()
    Ai = np.linalg.inv(Ad)
    rng = np.random.default_rng(3)
    n = Ad.shape[0]
    E1 = (rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n))) / np.sqrt(n)
    E2 = (rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n))) / np.sqrt(n)
    p1 = lambda r: Ai @ (r + 1e-3 * (E1 @ r))
    p2 = lambda r: p1(r) + 1e-11 * (Ai @ (E2 @ r))
    b = rng.standard_normal(n) + 1j * rng.standard_normal(n)
    res = mpgmres.solve(A, [p1, p2], b, tol=1e-12, maxit=30, keep_basis=True)
    assert res.status == "ok"
    assert res.Z.shape[1] == res.iterations  # one accepted direction per iteration
    assert res.rel_res_explicit < 10 * max(res.rel_res_implicit, 1e-14)


def test_zero_rhs():
    P, b = _setup()
    res = P.solve(np.zeros_like(b), tol=1e-8)
    assert res.iterations == 0 and np.all(res.x == 0)


def test_solution_matches_direct():
    k, n, N = 20.0, 32, 4
    P = solver.Problem(k, n, N)
    b = P.rhs(np.array([[0.5, 0.5, 0.05, 1.0, 0.0]]))
    res = P.solve(b, tol=1e-10)
    x = direct.solve(P.A, b, n)
    assert res.converged and res.rel_res_explicit < 1e-9
    assert np.linalg.norm(res.x - x) / np.linalg.norm(x) < 1e-7


def test_multipreconditioning_helps():
    """Section 4's qualitative finding: the two double sweeps LRL+BTB need fewer iterations
    than LRL alone."""
    k, n, N = 40.0, 64, 8
    one = solver.Problem(k, n, N, "LR")
    two = solver.Problem(k, n, N, "LR+BT")
    b = one.rhs(np.array([[0.5, 0.5, 0.05, 1.0, 0.0]]))
    assert two.solve(b, 1e-6).iterations < one.solve(b, 1e-6).iterations
