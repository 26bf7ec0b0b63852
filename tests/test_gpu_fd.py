"""GPU parity of the five-point mode (hh_opts.discretization = HH_DISC_FD: the paper's
finite differences and overlapping Robin-exchange strips, Section 4) against the oracle's FD
mode (oracle/fd.py), on the same seeded inputs.

Tolerances: the operator and the load vector are a few FP64 operations per entry (1e-13
relative); the sweeps use Gauss-Jordan inverses of the subdomain line blocks against the
oracle's banded LU, both FP64 (1e-10 relative, as for the P1 sweeps); solves take the oracle's
iteration count and its solution to 1e-10.
"""
import numpy as np
import pytest

import hh_inputs
import paper_2408_11929_gb300 as hh
from oracle import fd, fem

pytestmark = pytest.mark.gpu

# (k, n, strips): several strips with interior subdomains, two strips (both of R + 2 lines), one
# strip (the whole square), and a non-power-of-two line count
CASES = [(20.0, 32, 4), (15.0, 40, 5), (30.0, 48, 2), (12.0, 16, 1)]


@pytest.fixture(scope="module", autouse=True)
def built():
    import __graft_entry__
    __graft_entry__.build()


def rel(a, b):
    return np.linalg.norm(np.ravel(a) - np.ravel(b)) / np.linalg.norm(np.ravel(b))


def handle(k, n, N, dirs="LR+RL+BT+TB", **kw):
    return hh.Handle(k, n, N, dirs, discretization=hh.HH_DISC_FD, **kw)


@pytest.mark.parametrize("k,n,N", CASES)
def test_fd_operator(k, n, N):
    A = fd.global_matrix(k, n)
    x = hh_inputs.random_vector(A.shape[0], 3, seed=5)
    with handle(k, n, N) as h:
        y = h.apply_operator(np.ascontiguousarray(x.ravel()), 3).reshape(3, -1)
    for c in range(3):
        assert rel(y[c], A @ x[c]) < 1e-13


def test_fd_load_vector():
    k, n, N = 20.0, 32, 4
    src = np.array([[0.3, 0.6, 0.05, 1.0, 0.0], [0.71, 0.22, 0.08, -0.5, 2.0]])
    ref = fd.load_vector(n, fem.gaussian_source(n, src))
    with handle(k, n, N) as h:
        b = h.assemble_rhs(src)
    assert rel(b, ref) < 1e-13


@pytest.mark.parametrize("k,n,N", CASES)
@pytest.mark.parametrize("double", [True, False])
def test_fd_preconditioner(k, n, N, double):
    m2 = (n + 1) ** 2
    r = hh_inputs.random_vector(m2, 2, seed=6)
    with handle(k, n, N, single_sweep=0 if double else 1) as h:
        for d in fd.DIRECTIONS:
            sw = fd.OverlapSweeper(k, n, N, d)
            z = h.apply_preconditioner(d, np.ascontiguousarray(r.ravel()), 2).reshape(2, -1)
            for c in range(2):
                assert rel(z[c], sw.apply(r[c], double)) < 1e-10, (d, c)


@pytest.mark.parametrize("dirs,double", [("LR+RL+BT+TB", True), ("LR+BT", True), ("BT", True),
                                         ("LR+RL", False), ("LR+RL+BT+TB", False)])
def test_fd_solve_matches_oracle(dirs, double):
    """Table 1's combinations (double sweeps LRL, LRL+BTB and four directions; single sweeps
    LR+RL and LR+BT+RL+TB) with the paper's source: the oracle's iterations and solution."""
    k, n, N = 20.0, 32, 4
    P = fd.FDProblem(k, n, N, dirs, double)
    b = P.paper_rhs()
    ref = P.solve(b, tol=1e-8)
    with handle(k, n, N, dirs, single_sweep=0 if double else 1) as h:
        x, res = h.solve(b, tol=1e-8)
    assert res.status == hh.HH_OK
    assert res.iterations == ref.iterations
    assert rel(x, ref.x) < 1e-10
    assert res.rel_res_explicit < 1e-8


def test_fd_one_strip_is_exact():
    k, n = 12.0, 16
    P = fd.FDProblem(k, n, 1, "BT")
    b = P.paper_rhs()
    with handle(k, n, 1, "BT") as h:
        x, res = h.solve(b, tol=1e-10)
    assert res.status == hh.HH_OK and res.iterations == 1
    assert res.rel_res_explicit < 1e-12
