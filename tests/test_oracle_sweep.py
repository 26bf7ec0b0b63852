"""Pins of the oracle's strips and sweeps.

* one strip: the impedance-modified strip matrix is A itself, so the sweep is an exact
  solve and MPGMRES stops after one iteration;
* exact Schur complements as transmission blocks make the double sweep an exact block LU
  solve (Section 2: exact transparent conditions give a nilpotent iteration);
* the preconditioner formed explicitly, M = (D + L) D^{-1} (D + U), inverts the sweep;
* the square's symmetries (transpose, half-turn) map the BT sweep onto the other three;
* the factor cache changes nothing.
"""
import numpy as np
import pytest

from oracle import fem, mpgmres, solver, sweep


def _rhs(n, seed=0):
    rng = np.random.default_rng(seed)
    return rng.standard_normal((n + 1) ** 2) + 1j * rng.standard_normal((n + 1) ** 2)


def _transpose(n):
    m = n + 1
    i, j = np.meshgrid(np.arange(m), np.arange(m), indexing="xy")
    return (i * m + j).ravel()          # node (i, j) -> (j, i)


def _halfturn(n):
    return np.arange((n + 1) ** 2)[::-1]


@pytest.mark.parametrize("d", sweep.DIRECTIONS)
def test_one_strip_is_A(d):
    k, n = 15.0, 12
    A, *_ = fem.global_system(k, n)
    D, glob = sweep.strip_matrix(k, n, 0, n, sweep.orientation(d), 0)
    assert abs(D - A[glob][:, glob]).max() == 0


def test_one_strip_one_iteration():
    k, n = 15.0, 16
    P = solver.Problem(k, n, 1)
    b = P.rhs(np.array([[0.4, 0.6, 0.05, 1.0, 0.0]]))
    r = P.solve(b, 1e-10)
    assert r.iterations == 1 and r.rel_res_explicit < 1e-12


@pytest.mark.parametrize("d", sweep.DIRECTIONS)
def test_exact_schur_transmission_is_exact(d):
    k, n, N = 12.0, 12, 4
    A, *_ = fem.global_system(k, n)
    sw = sweep.Sweeper(A, k, n, N, d, strip_override=sweep.exact_schur_override(A, n, N, d))
    r = _rhs(n)
    z = sw.apply(r)
    assert np.linalg.norm(A @ z - r) / np.linalg.norm(r) < 1e-12
    res = mpgmres.solve(A, [lambda v: sw.apply(v)], r, tol=1e-10)
    assert res.iterations == 1


@pytest.mark.parametrize("d", sweep.DIRECTIONS)
@pytest.mark.parametrize("double", [True, False])
def test_explicit_preconditioner(d, double):
    k, n, N = 10.0, 8, 4
    A, *_ = fem.global_system(k, n)
    perm, DL, D, DU = sweep.block_operators(A, k, n, N, d)
    Mm = DL @ np.linalg.solve(D, DU) if double else DL
    sw = sweep.Sweeper(A, k, n, N, d)
    r = _rhs(n, 3)
    z = sw.apply(r, double)
    assert np.linalg.norm(Mm @ z[perm] - r[perm]) / np.linalg.norm(r) < 1e-12


def test_strip_blocks_structure():
    """Every strip visited before the last has the same matrix; its facing line block is
    A's bottom boundary block and every other row equals A's row."""
    k, n, N = 9.0, 16, 4
    A, *_ = fem.global_system(k, n)
    Ad = A.toarray()
    m = n + 1
    first = None
    for s, (a, b) in enumerate(sweep.strip_lines(n, N, "BT")):
        D, glob = sweep.strip_matrix(k, n, a, b, "row", sweep.far_side("BT", s, N))
        D = D.toarray()
        assert np.abs(D[:m, :m] - Ad[:m, :m]).max() == 0
        assert np.abs(D[m:, m:] - Ad[np.ix_(glob[m:], glob[m:])]).max() == 0
        if s < N - 1:
            first = D if first is None else first
            assert np.array_equal(D, first)
        else:
            assert D.shape[0] == (n // N + 1) * m


@pytest.mark.parametrize("double", [True, False])
def test_direction_symmetries(double):
    """LR = transpose o BT o transpose;  TB = half-turn o BT o half-turn;  RL = both."""
    k, n, N = 14.0, 16, 4
    A, *_ = fem.global_system(k, n)
    T, Q = _transpose(n), _halfturn(n)
    assert abs(A[T][:, T] - A).max() == 0 and abs(A[Q][:, Q] - A).max() == 0
    sw = {d: sweep.Sweeper(A, k, n, N, d, sweep.FactorCache(False)) for d in sweep.DIRECTIONS}
    r = _rhs(n, 5)
    bt = lambda v: sw["BT"].apply(v, double)
    zLR = sw["LR"].apply(r, double)
    zTB = sw["TB"].apply(r, double)
    zRL = sw["RL"].apply(r, double)
    ref = np.linalg.norm(zLR)
    assert np.linalg.norm(zLR - bt(r[T])[T]) / ref < 1e-12
    assert np.linalg.norm(zTB - bt(r[Q])[Q]) / ref < 1e-12
    TQ = T[Q]
    assert np.linalg.norm(zRL - bt(r[TQ])[np.argsort(TQ)]) / ref < 1e-12


def test_factor_cache_on_off():
    k, n, N = 11.0, 32, 4
    r = None
    xs = []
    for cache in (True, False):
        P = solver.Problem(k, n, N, cache=cache)
        if r is None:
            r = _rhs(n, 9)
        xs.append([p(r) for p in P.precs])
        if cache:
            assert P.cache.factorisations == 3
        else:
            assert P.cache.factorisations == 4 * N
    for a, b in zip(*xs):
        assert np.array_equal(a, b)


def test_strip_lines_partition():
    n, N = 32, 4
    for d in sweep.DIRECTIONS:
        lines = sweep.strip_lines(n, N, d)
        covered = sorted(j for a, b in lines for j in range(a, b + 1))
        assert covered == list(range(n + 1))
        assert lines[-1][1] - lines[-1][0] + 1 == n // N + 1
    with pytest.raises(ValueError):
        sweep.strip_lines(30, 4, "BT")
    with pytest.raises(ValueError):
        sweep.strip_lines(4, 4, "BT")
