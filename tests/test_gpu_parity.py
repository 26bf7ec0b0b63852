"""GPU parity: every entry point of the C ABI against the CPU oracle on the same seeded
inputs, element by element, at sizes the oracle finishes in seconds.

Tolerances.  FP64 paths: the stencil apply and the load vector are a few FP64 operations
per entry (1e-13 relative); the strip factors, sweeps and solutions differ from the
oracle only by rounding order of LAPACK's banded LU versus block Thomas with explicit
inverses, amplified by the conditioning of the strip blocks (1e-10 relative).  The
solution of the FP64 solver must match the oracle's to 1e-10 relative with the same
iteration count.  FP32 sweeps: complex64 factors (unit roundoff 6e-8) amplified by the
block conditioning give ~1e-4 relative agreement with the FP64 sweep; the FP32 solve must
reach the tolerance within the oracle's iterations + 2.
"""
import numpy as np
import pytest

import hh_inputs
import paper_2408_11929_gb300 as hh
from oracle import direct, fem, mpgmres, solver, sweep

pytestmark = pytest.mark.gpu

# (k, n, strips): several tiles, ragged line counts (R = 8, 16, 2), last strip R + 1
CASES = [(20.0, 32, 4), (15.0, 40, 5), (30.0, 48, 3), (12.0, 16, 8)]


@pytest.fixture(scope="module", autouse=True)
def built():
    import __graft_entry__
    __graft_entry__.build()


def rel(a, b):
    return np.linalg.norm(np.ravel(a) - np.ravel(b)) / np.linalg.norm(np.ravel(b))


@pytest.mark.parametrize("k,n,N", CASES)
def test_operator_apply(k, n, N):
    A, *_ = fem.global_system(k, n)
    x = hh_inputs.random_vector(A.shape[0], 3, seed=1)
    with hh.Handle(k, n, N) as h:
        y = h.apply_operator(np.ascontiguousarray(x.ravel()), 3).reshape(3, -1)
    for c in range(3):
        assert rel(y[c], A @ x[c]) < 1e-13


@pytest.mark.parametrize("k,n,N", CASES[:2])
def test_load_vector(k, n, N):
    src = np.array([[0.3, 0.6, 0.05, 1.0, 0.0], [0.71, 0.22, 0.08, -0.5, 2.0]])
    _, K, M, MG = fem.global_system(k, n)
    b_ref = fem.load_vector(n, M, MG, fem.gaussian_source(n, src))
    with hh.Handle(k, n, N) as h:
        b = h.assemble_rhs(src)
    assert rel(b, b_ref) < 1e-13


@pytest.mark.parametrize("k,n,N", [(20.0, 32, 4), (12.0, 16, 8)])
def test_strip_factors_fp64(k, n, N):
    """F_0 = D_bot^{-1}, F_j = (D_int - L F_{j-1} U)^{-1}, F_R = (D_top - L F_{R-1} U)^{-1}, with the
    line blocks taken from the oracle's global matrix (bottom line, an interior line, top line)."""
    A, *_ = fem.global_system(k, n)
    Ad = A.toarray()
    m, R = n + 1, n // N
    blk = lambda a, b: Ad[a * m:(a + 1) * m, b * m:(b + 1) * m]
    Dbot, Dint, Dtop = blk(0, 0), blk(1, 1), blk(n, n)
    L = blk(1, 0)
    U = blk(0, 1)
    ref = [np.linalg.inv(Dbot)]
    for j in range(1, R):
        ref.append(np.linalg.inv(Dint - L @ ref[-1] @ U))
    ref.append(np.linalg.inv(Dtop - L @ ref[-1] @ U))
    with hh.Handle(k, n, N) as h:
        for j in range(R + 1):
            assert rel(h.get_factor(j), ref[j]) < 1e-11, j


@pytest.mark.parametrize("k,n,N", [(20.0, 32, 4), (12.0, 16, 8), (100.0, 256, 16)])
def test_strip_factors_fp32_newton_schulz(k, n, N):
    """complex64 factors, all by Newton-Schulz on the tensor cores (F_0 from the Jacobi start,
    F_j from F_{j-1}, a block whose start diverges from the Jacobi start or the scaled
    adjoint); every one against the inverse of the oracle's Schur complement to complex64
    accuracy (the Schur complements have condition numbers near 6)."""
    A, *_ = fem.global_system(k, n)
    Ad = A.toarray() if n <= 64 else None
    m, R = n + 1, n // N
    As = A.tocsr()
    blk = lambda a, b: (Ad[a * m:(a + 1) * m, b * m:(b + 1) * m] if Ad is not None
                        else As[a * m:(a + 1) * m, b * m:(b + 1) * m].toarray())
    Dbot, Dint, Dtop = blk(0, 0), blk(1, 1), blk(n, n)
    L, U = blk(1, 0), blk(0, 1)
    ref = [np.linalg.inv(Dbot)]
    for j in range(1, R):
        ref.append(np.linalg.inv(Dint - L @ ref[-1] @ U))
    ref.append(np.linalg.inv(Dtop - L @ ref[-1] @ U))
    with hh.Handle(k, n, N, precision="fp32", twisted=0) as h:
        st = h.stats()
        assert st["ns_blocks"] == R + 1 and st["ns_iterations"] <= 16 * st["ns_blocks"]
        for j in range(R + 1):
            assert rel(h.get_factor(j), ref[j]) < 2e-5, j


@pytest.mark.parametrize("k,n,N", [(20.0, 32, 4), (30.0, 40, 8), (100.0, 256, 16)])
def test_twisted_strip_blocks(k, n, N):
    """The blocks of the twisted strip solves against dense references from the oracle's
    matrix: G_{R-1} = D_int^{-1}, G_j = (D_int - U G_{j+1} L)^{-1} down to j = q + 1 (q = R // 2),
    M = (D_int - L F_{q-1} U - U G_{q+1} L)^{-1} (F the block-Thomas inverses), and Z_0 =
    T^{-1}[0, R-1] U with T the strip matrix of lines 0..R-1; complex64 Newton-Schulz inverses,
    to 1e-4 relative (these sub-strips have no absorbing end, their inverses are larger)."""
    A, *_ = fem.global_system(k, n)
    As = A.tocsr()
    m, R = n + 1, n // N
    q = R // 2
    blk = lambda a, b: As[a * m:(a + 1) * m, b * m:(b + 1) * m].toarray()
    Dbot, Dint = blk(0, 0), blk(1, 1)
    L, U = blk(1, 0), blk(0, 1)
    F = [np.linalg.inv(Dbot)]
    for j in range(1, R):
        F.append(np.linalg.inv(Dint - L @ F[-1] @ U))
    G = {R - 1: np.linalg.inv(Dint)}
    for j in range(R - 2, q, -1):
        G[j] = np.linalg.inv(Dint - U @ G[j + 1] @ L)
    M = np.linalg.inv(Dint - L @ F[q - 1] @ U - U @ G[q + 1] @ L)
    T = As[:R * m, :R * m].toarray()
    Z0 = np.linalg.solve(T, np.vstack([np.zeros(((R - 1) * m, m)), U]))[:m]
    with hh.Handle(k, n, N, precision="fp32", twisted=1) as h:
        nb = h.stats()["factor_blocks"]
        base = nb - 2 - (R - 1 - q)
        for j in range(q + 1, R):
            assert rel(h.get_factor(base + j - q - 1), G[j]) < 1e-4, j
        assert rel(h.get_factor(nb - 2), M) < 1e-4
        assert rel(h.get_factor(nb - 1), Z0) < 1e-4


@pytest.mark.parametrize("k,n,N", CASES)
@pytest.mark.parametrize("double", [True, False])
def test_preconditioner_fp64(k, n, N, double):
    A, *_ = fem.global_system(k, n)
    r = hh_inputs.random_vector(A.shape[0], 2, seed=2)
    with hh.Handle(k, n, N, single_sweep=0 if double else 1) as h:
        for d in sweep.DIRECTIONS:
            sw = sweep.Sweeper(A, k, n, N, d)
            z = h.apply_preconditioner(d, np.ascontiguousarray(r.ravel()), 2).reshape(2, -1)
            for c in range(2):
                assert rel(z[c], sw.apply(r[c], double)) < 1e-10, (d, c)


@pytest.mark.parametrize("k,n,N", CASES[:2])
def test_preconditioner_fp32(k, n, N):
    A, *_ = fem.global_system(k, n)
    r = hh_inputs.random_vector(A.shape[0], 4, seed=3)
    with hh.Handle(k, n, N, precision="fp32") as h:
        for d in sweep.DIRECTIONS:
            sw = sweep.Sweeper(A, k, n, N, d)
            z = h.apply_preconditioner(d, np.ascontiguousarray(r.ravel()), 4).reshape(4, -1)
            for c in range(4):
                assert rel(z[c], sw.apply(r[c])) < 2e-4, (d, c)


@pytest.mark.parametrize("dirs", ["LR+RL+BT+TB", "LR+BT", "BT", "RL+BT+TB", "TB+LR"])
def test_solve_fp64_matches_oracle(dirs):
    k, n, N = 20.0, 32, 4
    P = solver.Problem(k, n, N, dirs)
    src = hh_inputs.centre_source()
    b = P.rhs(src)
    # the handle orders preconditioners LR, RL, BT, TB; the oracle keeps the string order
    order = [d for d in ("LR", "RL", "BT", "TB") if d in dirs.split("+")]
    ref = solver.Problem(k, n, N, "+".join(order)).solve(b, tol=1e-8)
    with hh.Handle(k, n, N, dirs) as h:
        x, res = h.solve(b, tol=1e-8)
    assert res.status == hh.HH_OK
    assert res.iterations == ref.iterations
    assert rel(x, ref.x) < 1e-10
    assert res.rel_res_explicit < 1e-8
    assert abs(res.rel_res_implicit - ref.history[-1]) < 1e-3 * ref.history[-1]


def test_solve_batch_matches_single_solves():
    k, n, N = 25.0, 48, 4
    srcs = hh_inputs.random_sources(3, seed=7, complex_amp=True)
    P = solver.Problem(k, n, N)
    B = np.stack([P.rhs(s) for s in srcs])
    with hh.Handle(k, n, N) as h:
        X, res = h.solve_batch(np.ascontiguousarray(B.ravel()), 3, tol=1e-8)
        X = X.reshape(3, -1)
        for r in range(3):
            ref = P.solve(B[r], tol=1e-8)
            assert res[r].status == hh.HH_OK
            assert res[r].iterations == ref.iterations
            assert rel(X[r], ref.x) < 1e-10


def test_device_pointers_torch():
    torch = pytest.importorskip("torch")
    k, n, N = 20.0, 32, 4
    P = solver.Problem(k, n, N)
    b = P.rhs(hh_inputs.centre_source())
    ref = P.solve(b, tol=1e-8)
    bt = torch.from_numpy(b).cuda()
    with hh.Handle(k, n, N) as h:
        xt, res = h.solve(bt, tol=1e-8)
        assert xt.is_cuda
        assert res.iterations == ref.iterations
        assert rel(xt.cpu().numpy(), ref.x) < 1e-10
        bd = torch.zeros(b.size, dtype=torch.complex128, device="cuda")
        h.assemble_rhs(hh_inputs.centre_source(), out=bd)
        assert rel(bd.cpu().numpy(), b) < 1e-13


def test_one_strip_is_exact():
    k, n = 18.0, 24
    P = solver.Problem(k, n, 1)
    b = P.rhs(hh_inputs.centre_source())
    with hh.Handle(k, n, 1) as h:
        x, res = h.solve(b, tol=1e-10)
    assert res.status == hh.HH_OK and res.iterations == 1
    assert rel(x, direct.solve(P.A, b, n)) < 1e-10


def test_zero_rhs():
    with hh.Handle(10.0, 16, 4) as h:
        x, res = h.solve(np.zeros(17 * 17, dtype=np.complex128), tol=1e-8)
    assert res.status == hh.HH_OK and res.iterations == 0
    assert np.all(x == 0)


def test_maxit_reports_noconv():
    k, n, N = 20.0, 32, 4
    P = solver.Problem(k, n, N)
    b = P.rhs(hh_inputs.centre_source())
    ref = P.solve(b, tol=1e-12, maxit=3)
    with hh.Handle(k, n, N, maxit=3) as h:
        x, res = h.solve(b, tol=1e-12)
    assert res.status == hh.HH_ENOCONV and res.iterations == 3
    assert rel(x, ref.x) < 1e-10


def test_bounded_wait_times_out_and_context_survives():
    """A cycle budget of 1 makes the first grid barrier of the strip setup give up; the
    kernel returns, the call reports HH_ETIMEOUT and the device stays usable."""
    with pytest.raises(hh.HHError) as e:
        hh.Handle(10.0, 16, 4, timeout_cycles=1)
    assert e.value.status == hh.HH_ETIMEOUT
    with hh.Handle(10.0, 16, 4) as h:
        x, res = h.solve(h.assemble_rhs(hh_inputs.centre_source()), tol=1e-8)
    assert res.status == hh.HH_OK


def test_submit_poll_matches_solve():
    import time
    k, n, N = 20.0, 32, 4
    srcs = hh_inputs.random_sources(4, seed=11)
    with hh.Handle(k, n, N) as h:
        bs = [h.assemble_rhs(s) for s in srcs]
        xs = [np.zeros_like(b) for b in bs]
        tickets = [h.submit(b, x, tol=1e-8) for b, x in zip(bs, xs)]
        done = {}
        t0 = time.time()
        while len(done) < len(tickets) and time.time() - t0 < 60:
            for t in tickets:
                if t not in done:
                    st, res = h.poll(t)
                    if st != hh.HH_EPENDING:
                        done[t] = (st, res)
            time.sleep(0.001)
        assert len(done) == len(tickets)
        for b, x, t in zip(bs, xs, tickets):
            xr, rr = h.solve(b, tol=1e-8)
            assert done[t][0] == hh.HH_OK
            assert done[t][1].iterations == rr.iterations
            assert rel(x, xr) < 1e-12


def test_fp32_sweeps_solve():
    k, n, N = 40.0, 64, 4
    P = solver.Problem(k, n, N)
    b = P.rhs(hh_inputs.centre_source())
    ref = P.solve(b, tol=1e-6)
    tight = P.solve(b, tol=1e-10)
    with hh.Handle(k, n, N, precision="fp32") as h:
        x, res = h.solve(b, tol=1e-6)
    assert res.status == hh.HH_OK
    assert res.iterations <= ref.iterations + 2
    assert res.rel_res_explicit < 1.5e-6
    assert rel(x, tight.x) < 1e-5


@pytest.mark.parametrize("dirs", ["LR+RL+BT+TB", "LR+BT"])
def test_single_pass_gram_schmidt_matches_oracle(dirs):
    """gs_passes = 1: one classical Gram-Schmidt pass (Section 3's inner-product count),
    against the oracle run with the same single pass."""
    k, n, N = 30.0, 48, 4
    P = solver.Problem(k, n, N, dirs)
    b = P.rhs(hh_inputs.centre_source())
    ref = P.solve(b, tol=1e-8, gs_passes=1)
    with hh.Handle(k, n, N, dirs, gs_passes=1) as h:
        x, res = h.solve(b, tol=1e-8)
    assert res.status == hh.HH_OK and res.iterations == ref.iterations
    assert rel(x, ref.x) < 1e-10


def test_continuous_batching_matches_alone():
    """Requests with mixed tolerances arrive while others are mid-solve and share two slots
    (serve_slots = 2, five requests): each result equals the same request solved alone."""
    import time
    k, n, N = 25.0, 48, 4
    srcs = hh_inputs.random_sources(5, seed=21, complex_amp=True)
    tols = [1e-6, 1e-10, 1e-8, 1e-7, 1e-9]
    with hh.Handle(k, n, N, serve_slots=2) as h:
        bs = [h.assemble_rhs(s) for s in srcs]
        alone = [h.solve(b, tol=t) for b, t in zip(bs, tols)]
        xs = [np.zeros_like(b) for b in bs]
        tickets = [h.submit(bs[0], xs[0], tol=tols[0])]
        time.sleep(0.05)  # the first request is iterating when the others arrive
        tickets += [h.submit(b, x, tol=t) for b, x, t in zip(bs[1:], xs[1:], tols[1:])]
        done = {}
        t0 = time.time()
        while len(done) < len(tickets) and time.time() - t0 < 120:
            for t in tickets:
                if t not in done:
                    st, res = h.poll(t)
                    if st != hh.HH_EPENDING:
                        done[t] = (st, res)
            time.sleep(0.001)
    assert len(done) == len(tickets)
    for (xa, ra), x, t, tol in zip(alone, xs, tickets, tols):
        st, res = done[t]
        assert st == hh.HH_OK and res.iterations == ra.iterations
        assert res.rel_res_explicit < tol
        assert rel(x, xa) < 1e-10


def test_batch_zero_and_nonzero_columns():
    """A zero right-hand side inside a batch finishes at admission with x = 0 while the
    other columns iterate to the oracle's iteration count."""
    k, n, N = 20.0, 32, 4
    P = solver.Problem(k, n, N)
    b = P.rhs(hh_inputs.centre_source())
    ref = P.solve(b, tol=1e-8)
    B = np.stack([np.zeros_like(b), b, np.zeros_like(b)])
    with hh.Handle(k, n, N) as h:
        X, res = h.solve_batch(np.ascontiguousarray(B.ravel()), 3, tol=1e-8)
    X = X.reshape(3, -1)
    assert res[0].iterations == 0 and res[2].iterations == 0 and np.all(X[0] == 0) and np.all(X[2] == 0)
    assert res[1].iterations == ref.iterations and rel(X[1], ref.x) < 1e-10


@pytest.mark.parametrize("k,n,N", [(20.0, 32, 4), (15.0, 40, 5), (60.0, 256, 8)])
def test_tensor_core_sweeps(k, n, N):
    """complex64 sweeps on the tensor cores (TF32 operands split hi + lo, three products, FP32
    accumulation), with the twisted strip solves (grouped steps) and with block Thomas (line
    steps), against the CUDA-core complex64 sweeps and the FP64 oracle sweep."""
    A, *_ = fem.global_system(k, n)
    r = hh_inputs.random_vector(A.shape[0], 4, seed=5)
    errs = {}
    with hh.Handle(k, n, N, precision="fp32", tensor_cores=1) as ht, \
            hh.Handle(k, n, N, precision="fp32", tensor_cores=1, twisted=0) as ht0, \
            hh.Handle(k, n, N, precision="fp32", tensor_cores=0) as hc:
        assert ht.stats()["tensor_cores"] == 1 and hc.stats()["tensor_cores"] == 0
        for d in sweep.DIRECTIONS:
            sw = sweep.Sweeper(A, k, n, N, d)
            zt = ht.apply_preconditioner(d, np.ascontiguousarray(r.ravel()), 4).reshape(4, -1)
            zt0 = ht0.apply_preconditioner(d, np.ascontiguousarray(r.ravel()), 4).reshape(4, -1)
            zc = hc.apply_preconditioner(d, np.ascontiguousarray(r.ravel()), 4).reshape(4, -1)
            assert ht.stats()["twisted"] == 1 and ht0.stats()["twisted"] == 0
            for c in range(4):
                ref = sw.apply(r[c])
                errs[(d, c)] = (rel(zt[c], ref), rel(zt0[c], ref), rel(zc[c], ref))
    worst_t = max(e[0] for e in errs.values())
    worst_t0 = max(e[1] for e in errs.values())
    worst_c = max(e[2] for e in errs.values())
    print(f"tensor-core vs oracle {worst_t:.2e} (twisted) {worst_t0:.2e} (Thomas), CUDA-core {worst_c:.2e}")
    assert worst_c < 2e-4
    assert worst_t < 2e-4 and worst_t0 < 2e-4


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_step_graphs_replayed_and_equal_to_eager(precision):
    """Every Arnoldi step is captured as a CUDA graph (including the cooperative block QR) and
    replayed; the result equals the eager solve (use_graph = 0) to rounding."""
    k, n, N = 30.0, 48, 4
    src = hh_inputs.centre_source()
    with hh.Handle(k, n, N, precision=precision) as h:
        b = h.assemble_rhs(src)
        xg, rg = h.solve(b, tol=1e-8)
        st = h.stats()
    with hh.Handle(k, n, N, precision=precision, use_graph=0) as h:
        xe, re_ = h.solve(b, tol=1e-8)
    assert st["step_graphs"] >= 1 and st["step_graph_fallback"] == 0
    assert rg.iterations == re_.iterations
    assert rel(xg, xe) < (1e-12 if precision == "fp64" else 1e-5)


@pytest.mark.parametrize("cand", range(21))
def test_tensor_core_step_candidates(cand):
    """Every candidate of the tensor-core step's autotuner (three tile shapes; K split by a
    reduction kernel or in a thread-block cluster) gives the complex64 sweep within the bar.
    8 strips x 4 columns: 32 columns, a partial tile of every shape.  Block Thomas, whose
    strip-solve steps are the line steps the candidates apply to."""
    k, n, N = 60.0, 256, 8
    A, *_ = fem.global_system(k, n)
    r = hh_inputs.random_vector(A.shape[0], 4, seed=9)
    with hh.Handle(k, n, N, precision="fp32", autotune=-(1 + cand), twisted=0) as h:
        for d in ("BT", "LR"):
            sw = sweep.Sweeper(A, k, n, N, d)
            z = h.apply_preconditioner(d, np.ascontiguousarray(r.ravel()), 4).reshape(4, -1)
            st = h.stats()
            assert st["tc_bnc"] == (64, 32, 128)[cand // 7] and st["tc_cluster"] == int(cand % 7 >= 4)
            for c in range(4):
                assert rel(z[c], sw.apply(r[c])) < 2e-4, (d, c)


@pytest.mark.parametrize("variant", [0, 3, 4, 6])
def test_tensor_core_128_column_tiles(variant):
    """The 128-column tile shape over two column tiles (32 strips x 8 columns = 256 columns),
    K split by the reduction kernel or in a cluster, against the oracle sweep."""
    k, n, N = 60.0, 256, 32
    A, *_ = fem.global_system(k, n)
    r = hh_inputs.random_vector(A.shape[0], 8, seed=10)
    with hh.Handle(k, n, N, precision="fp32", autotune=-(1 + 14 + variant), twisted=0) as h:
        for d in ("TB", "RL"):
            sw = sweep.Sweeper(A, k, n, N, d)
            z = h.apply_preconditioner(d, np.ascontiguousarray(r.ravel()), 8).reshape(8, -1)
            assert h.stats()["tc_bnc"] == 128
            for c in range(8):
                assert rel(z[c], sw.apply(r[c])) < 2e-4, (d, c)


@pytest.mark.parametrize("precision,ncols", [("fp64", 2), ("fp64", 4), ("fp32", 4), ("fp32", 8)])
@pytest.mark.parametrize("single", [0, 1])
def test_fused_interface_chains(precision, ncols, single):
    """The interface chains (N-2 and N-1 dependent strip-to-strip steps of Section 2's sweep)
    run as one cooperative launch each, factor block kept in shared memory, grid barriers
    between the steps: the sweep equals the two-launches-per-step form to rounding and the
    oracle's sweep within the bar, with fewer launches.  16 strips: chains of 14 and 15 steps;
    257 node rows spread raggedly over one CTA per SM."""
    k, n, N = 40.0, 256, 16
    A, *_ = fem.global_system(k, n)
    r = hh_inputs.random_vector(A.shape[0], ncols, seed=11)
    rr = np.ascontiguousarray(r.ravel())
    bar = 1e-10 if precision == "fp64" else 2e-4
    # both handles run the same tensor-core candidate (the autotuner could give them forms
    # with different launches per wide step), so the launch counts differ by the fusion only
    # the chains exist in interface form 0 (form 1 replaces them by scans)
    with hh.Handle(k, n, N, precision=precision, single_sweep=single, autotune=0, interface_form=0) as hf, \
            hh.Handle(k, n, N, precision=precision, single_sweep=single, fuse_chains=0, autotune=0,
                      interface_form=0) as hu:
        for d in sweep.DIRECTIONS:
            hf.apply_preconditioner(d, rr, ncols)
            hu.apply_preconditioner(d, rr, ncols)
            hf.reset_stats()
            hu.reset_stats()
            zf = hf.apply_preconditioner(d, rr, ncols).reshape(ncols, -1)
            zu = hu.apply_preconditioner(d, rr, ncols).reshape(ncols, -1)
            lf, lu = hf.stats()["kernel_launches"], hu.stats()["kernel_launches"]
            assert lf < lu, (lf, lu)
            assert rel(zf, zu) < (1e-12 if precision == "fp64" else 1e-4)
            sw = sweep.Sweeper(A, k, n, N, d)
            for c in range(ncols):
                assert rel(zf[c], sw.apply(r[c], not single)) < bar, (d, c)


def test_fused_interface_chain_many_rows():
    """n = 1536: 1537 node rows over one CTA per SM puts more rows on a CTA than it has warps
    (each warp takes several rows); the fused chains equal the per-step form to rounding."""
    k, n, N = 600.0, 1536, 16
    rr = np.ascontiguousarray(hh_inputs.random_vector((n + 1) ** 2, 4, seed=12).ravel())
    with hh.Handle(k, n, N, precision="fp32", autotune=0, interface_form=0) as hf, \
            hh.Handle(k, n, N, precision="fp32", autotune=0, fuse_chains=0, interface_form=0) as hu:
        for d in ("BT", "LR"):
            zf = hf.apply_preconditioner(d, rr, 4)
            zu = hu.apply_preconditioner(d, rr, 4)
            assert np.all(np.isfinite(zf))
            assert rel(zf, zu) < 1e-4


@pytest.mark.parametrize("autotune,twisted", [(0, 1), (0, 0), (-(1 + 7 + 5), 0), (-(1 + 14 + 0), 0)])
def test_overlapped_tensor_core_steps_equal_plain_order(autotune, twisted):
    """Programmatic dependent launch of the tensor-core steps (prologue and factor tiles of a
    step overlapping the end of the previous kernel) changes only the schedule: the sweeps
    are bit-identical to plain stream order and a whole solve agrees to rounding, for the
    default shape, a cluster candidate and the 128-column shape of the line steps (block
    Thomas), and for the grouped steps of the twisted strip solves."""
    k, n, N = 60.0, 256, 8
    rr = np.ascontiguousarray(hh_inputs.random_vector((n + 1) ** 2, 4, seed=13).ravel())
    src = hh_inputs.centre_source()
    with hh.Handle(k, n, N, precision="fp32", autotune=autotune, twisted=twisted) as ho, \
            hh.Handle(k, n, N, precision="fp32", autotune=autotune, twisted=twisted, overlap_steps=0) as hp:
        for d in sweep.DIRECTIONS:
            assert np.array_equal(ho.apply_preconditioner(d, rr, 4), hp.apply_preconditioner(d, rr, 4)), d
        b = ho.assemble_rhs(src)
        xo, ro = ho.solve(b, tol=1e-6)
        xp, rp = hp.solve(b, tol=1e-6)
    assert ro.iterations == rp.iterations and rel(xo, xp) < 1e-12


@pytest.mark.parametrize("twisted", [0, 1])
def test_tensor_map_cache_turnover(twisted):
    """The tensor maps of the sweep arrays are cached in a ring keyed by (array, columns,
    tile shape); sweeps over many column counts on one handle turn the ring over several
    times, and every sweep still equals the oracle's (a step whose two maps were looked up
    across an eviction would read the wrong array)."""
    k, n, N = 20.0, 64, 4
    A, *_ = fem.global_system(k, n)
    sw = sweep.Sweeper(A, k, n, N, "LR")
    with hh.Handle(k, n, N, precision="fp32", autotune=-(1 + 7 + 5), twisted=twisted) as h:
        for ncols in (2, 4, 6, 8, 10, 12, 14, 16, 2, 4):
            r = hh_inputs.random_vector(A.shape[0], ncols, seed=20 + ncols)
            z = h.apply_preconditioner("LR", np.ascontiguousarray(r.ravel()), ncols).reshape(ncols, -1)
            for c in range(ncols):
                assert rel(z[c], sw.apply(r[c])) < 2e-4, (ncols, c)


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
@pytest.mark.parametrize("k,n,N", CASES + [(10.0, 16, 2), (25.0, 64, 16), (20.0, 36, 6)])
@pytest.mark.parametrize("double", [True, False])
def test_interface_scans_and_block_column_corrections(precision, k, n, N, double):
    """Interface form 1 (prefix-doubling scans of the strip-to-strip recurrences, interior
    corrections as one grouped step with stored block columns of the strip inverse) against
    the oracle's sweep and against interface form 0 (chains and block-Thomas corrections):
    the same sweep up to rounding.  N = 2, 3, 5, 6 strips cover scans of 0, 1 and ragged
    numbers of levels; 4 columns (the tensor cores for complex64) and 3 (the CUDA cores)."""
    A, *_ = fem.global_system(k, n)
    for ncols in (4, 3):
        r = hh_inputs.random_vector(A.shape[0], ncols, seed=30 + ncols)
        rr = np.ascontiguousarray(r.ravel())
        bar = 1e-10 if precision == "fp64" else 2e-4
        with hh.Handle(k, n, N, precision=precision, single_sweep=0 if double else 1) as h1, \
                hh.Handle(k, n, N, precision=precision, single_sweep=0 if double else 1, interface_form=0) as h0:
            assert h1.stats()["sweep_steps"] < h0.stats()["sweep_steps"] or N <= 2
            for d in sweep.DIRECTIONS:
                z1 = h1.apply_preconditioner(d, rr, ncols).reshape(ncols, -1)
                z0 = h0.apply_preconditioner(d, rr, ncols).reshape(ncols, -1)
                assert rel(z1, z0) < (1e-11 if precision == "fp64" else 1e-4), (d, ncols)
                sw = sweep.Sweeper(A, k, n, N, d)
                for c in range(ncols):
                    assert rel(z1[c], sw.apply(r[c], double)) < bar, (d, c, ncols)


BCR_CASES = [(20.0, 32, 4), (30.0, 48, 3), (25.0, 64, 16), (20.0, 36, 6), (12.0, 16, 8)]


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
@pytest.mark.parametrize("k,n,N", BCR_CASES)
def test_cyclic_reduction_depths(precision, k, n, N):
    """Strip solves by block cyclic reduction of every usable depth d (R divisible by 2^d):
    the double and the single sweep equal the oracle's (banded LU strip solves) and the
    block-Thomas form (d = 0) up to rounding; fewer dependent steps for d >= 1 when R >= 4.
    Columns 4 (tensor cores for complex64) and 3 (CUDA cores)."""
    R = n // N
    dmax = 0
    while R % (2 << dmax) == 0:
        dmax += 1
    A, *_ = fem.global_system(k, n)
    bar = 1e-10 if precision == "fp64" else 2e-4
    for d in range(1, dmax + 1):
        for ncols in (4, 3):
            r = hh_inputs.random_vector(A.shape[0], ncols, seed=40 + d + ncols)
            rr = np.ascontiguousarray(r.ravel())
            for single in (0, 1):
                with hh.Handle(k, n, N, precision=precision, bcr_depth=d, single_sweep=single) as hd, \
                        hh.Handle(k, n, N, precision=precision, bcr_depth=0, twisted=0, single_sweep=single) as h0:
                    for dd in ("BT", "LR", "TB", "RL"):
                        zd = hd.apply_preconditioner(dd, rr, ncols).reshape(ncols, -1)
                        z0 = h0.apply_preconditioner(dd, rr, ncols).reshape(ncols, -1)
                        assert hd.stats()["bcr_depth"] == d
                        assert rel(zd, z0) < (1e-11 if precision == "fp64" else 1e-4), (d, dd, ncols, single)
                        sw = sweep.Sweeper(A, k, n, N, dd)
                        for c in range(ncols):
                            assert rel(zd[c], sw.apply(r[c], not single)) < bar, (d, dd, c, single)
                    if R >= 4:
                        assert hd.stats()["sweep_steps"] < h0.stats()["sweep_steps"]


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_cyclic_reduction_autotuned_solve(precision):
    """bcr_depth = -1: every usable depth is stored and the fastest is picked by timing whole
    sweeps; the solve equals the oracle's (FP64: same iterations, 1e-10; FP32: within the
    oracle's iterations + 2)."""
    k, n, N = 30.0, 64, 4
    P = solver.Problem(k, n, N)
    b = P.rhs(hh_inputs.centre_source())
    tol = 1e-8 if precision == "fp64" else 1e-6
    ref = P.solve(b, tol=tol)
    with hh.Handle(k, n, N, precision=precision, bcr_depth=-1) as h:
        x, res = h.solve(b, tol=tol)
        st = h.stats()
    assert 0 <= st["bcr_depth"] <= 4
    assert res.status == hh.HH_OK
    if precision == "fp64":
        assert res.iterations == ref.iterations and rel(x, ref.x) < 1e-10
    else:
        assert res.iterations <= ref.iterations + 2 and res.rel_res_explicit < 1.5e-6


def test_cyclic_reduction_solve_fp64_matches_oracle():
    """A whole FP64 solve with depth-3 cyclic reduction (R = 8): the oracle's iteration count
    and solution to 1e-10."""
    k, n, N = 20.0, 32, 4
    P = solver.Problem(k, n, N)
    b = P.rhs(hh_inputs.centre_source())
    ref = P.solve(b, tol=1e-8)
    with hh.Handle(k, n, N, precision="fp64", bcr_depth=3) as h:
        x, res = h.solve(b, tol=1e-8)
    assert res.status == hh.HH_OK and res.iterations == ref.iterations
    assert rel(x, ref.x) < 1e-10


# (k, n, strips): R = 8, 16, 4, 6, 5 (odd: the ends meet unevenly), 45 (two strips), 32
TWIST_CASES = [(20.0, 32, 4), (30.0, 48, 3), (25.0, 64, 16), (20.0, 36, 6), (15.0, 40, 8), (30.0, 90, 2),
               (60.0, 256, 8)]


@pytest.mark.parametrize("k,n,N", TWIST_CASES)
def test_twisted_strip_solves(k, n, N):
    """The strip solves by the twisted block factorisation (both ends of every strip eliminated
    at once, meeting at line R/2; the last strip's extra line by its Schur complement after the
    interface corrections): the double and the single complex64 sweep equal block Thomas to
    1e-4 and the oracle's (banded LU in FP64) to the complex64 bar, in all four directions; an
    odd column count (CUDA-core kernels) keeps block Thomas; the chain is shorter."""
    A, *_ = fem.global_system(k, n)
    for ncols in (4, 2, 3):
        r = hh_inputs.random_vector(A.shape[0], ncols, seed=70 + ncols)
        rr = np.ascontiguousarray(r.ravel())
        for single in (0, 1):
            with hh.Handle(k, n, N, precision="fp32", twisted=1, single_sweep=single) as ht, \
                    hh.Handle(k, n, N, precision="fp32", twisted=0, single_sweep=single) as h0:
                for d in sweep.DIRECTIONS:
                    zt = ht.apply_preconditioner(d, rr, ncols).reshape(ncols, -1)
                    z0 = h0.apply_preconditioner(d, rr, ncols).reshape(ncols, -1)
                    assert ht.stats()["twisted"] == (1 if ncols % 2 == 0 else 0), ncols
                    assert rel(zt, z0) < 1e-4, (d, ncols, single)
                    sw = sweep.Sweeper(A, k, n, N, d)
                    for c in range(ncols):
                        assert rel(zt[c], sw.apply(r[c], not single)) < 2e-4, (d, c, single)
                if ncols % 2 == 0:
                    assert ht.stats()["sweep_steps"] < h0.stats()["sweep_steps"]


@pytest.mark.parametrize("k,n,N,ncols", [(20.0, 32, 4, 4), (60.0, 256, 8, 8), (30.0, 90, 2, 2)])
def test_twisted_strip_solves_persistent_and_bf16(k, n, N, ncols):
    """The twisted program in the one-launch persistent sweep equals its phase-by-phase launches
    (complex64 both, K slices summed in another order: 5e-5, the longer chains through the
    meeting line's Schur complement amplify it more than block Thomas does).  bf16 factor
    products keep block Thomas: the handle reports no twisted solves and the same sweep as a
    handle without them."""
    A, *_ = fem.global_system(k, n)
    r = hh_inputs.random_vector(A.shape[0], ncols, seed=80 + ncols)
    rr = np.ascontiguousarray(r.ravel())
    for single in (0, 1):
        with hh.Handle(k, n, N, precision="fp32", twisted=1, single_sweep=single, persistent=1) as hp, \
                hh.Handle(k, n, N, precision="fp32", twisted=1, single_sweep=single, persistent=0) as hl, \
                hh.Handle(k, n, N, precision="bf16", twisted=1, single_sweep=single) as hb, \
                hh.Handle(k, n, N, precision="bf16", twisted=0, single_sweep=single) as hb0:
            for d in sweep.DIRECTIONS:
                zp = hp.apply_preconditioner(d, rr, ncols).reshape(ncols, -1)
                zl = hl.apply_preconditioner(d, rr, ncols).reshape(ncols, -1)
                zb = hb.apply_preconditioner(d, rr, ncols).reshape(ncols, -1)
                zb0 = hb0.apply_preconditioner(d, rr, ncols).reshape(ncols, -1)
                assert hp.stats()["twisted"] == 1 and hb.stats()["twisted"] == 0
                assert rel(zp, zl) < 5e-5, (d, single)
                sw = sweep.Sweeper(A, k, n, N, d)
                for c in range(ncols):
                    ref = sw.apply(r[c], not single)
                    assert rel(zl[c], ref) < 2e-4, (d, c, single)
                    assert rel(zb[c], zb0[c]) < 1e-6, (d, c, single)


@pytest.mark.parametrize("twisted", [1, -1])
def test_twisted_solve(twisted):
    """A complex64 solve with the twisted strip solves (forced, or timed against block Thomas
    per column count): tol 1e-6 in explicit residual within the oracle's iterations + 2, the
    solution within 1e-4 of the oracle's."""
    k, n, N = 40.0, 128, 8
    P = solver.Problem(k, n, N)
    b = P.rhs(hh_inputs.centre_source())
    ref = P.solve(b, tol=1e-6)
    with hh.Handle(k, n, N, precision="fp32", twisted=twisted) as h:
        x, res = h.solve(b, tol=1e-6)
        st = h.stats()
    assert res.status == hh.HH_OK
    assert res.iterations <= ref.iterations + 2 and res.rel_res_explicit < 1.5e-6
    assert rel(x, ref.x) < 1e-4
    if twisted == 1:
        assert st["twisted"] == 1 and st["bcr_depth"] == 0
    else:
        assert st["twisted"] in (0, 1)


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
@pytest.mark.parametrize("dirs", ["LR+RL", "LR+RL+BT+TB"])
def test_single_sweep_combinations_solve(precision, dirs):
    """Table 1's single-sweep combinations LR+RL and LR+BT+RL+TB (forward sweeps only) as whole
    solves against the oracle's MPGMRES with the same forward-only preconditioners: FP64 the
    same iteration count and the solution to 1e-10; complex64 sweeps within the oracle's
    iterations + 2 at tol 1e-6."""
    k, n, N = 30.0, 64, 8
    P = solver.Problem(k, n, N, dirs, double=False)
    b = P.rhs(hh_inputs.centre_source())
    tol = 1e-8 if precision == "fp64" else 1e-6
    ref = P.solve(b, tol=tol)
    with hh.Handle(k, n, N, dirs, precision=precision, single_sweep=1) as h:
        x, res = h.solve(b, tol=tol)
    assert res.status == hh.HH_OK
    if precision == "fp64":
        assert res.iterations == ref.iterations
        assert rel(x, ref.x) < 1e-10
    else:
        assert res.iterations <= ref.iterations + 2 and res.rel_res_explicit < 1.5e-6
        assert rel(x, ref.x) < 1e-4


@pytest.mark.parametrize("k,n,N,ncols", [(20.0, 32, 4, 4), (40.0, 256, 16, 4), (60.0, 256, 8, 8), (30.0, 96, 3, 2)])
@pytest.mark.parametrize("bcr", [0, 2])
@pytest.mark.parametrize("form", [1, 2])
def test_persistent_sweep_equals_phase_launches(k, n, N, ncols, bcr, form):
    """The whole sweep as one persistent cooperative launch (every phase of the program, grid
    barriers between them, K split through an L2 buffer where a phase has few tiles) equals
    the same program launched phase by phase, and the oracle's sweep, for the double and the
    single sweep."""
    R = n // N
    if R % (1 << bcr):
        pytest.skip("depth needs R divisible by 2^d")
    A, *_ = fem.global_system(k, n)
    r = hh_inputs.random_vector(A.shape[0], ncols, seed=50 + ncols)
    rr = np.ascontiguousarray(r.ravel())
    for single in (0, 1):
        with hh.Handle(k, n, N, precision="fp32", bcr_depth=bcr, single_sweep=single, persistent=form) as hp, \
                hh.Handle(k, n, N, precision="fp32", bcr_depth=bcr, single_sweep=single, persistent=0) as hl:
            hp.apply_preconditioner("BT", rr, ncols)  # tuning runs outside the counted sweeps
            hl.apply_preconditioner("BT", rr, ncols)
            hp.reset_stats()
            hl.reset_stats()
            for d in sweep.DIRECTIONS:
                zp = hp.apply_preconditioner(d, rr, ncols).reshape(ncols, -1)
                zl = hl.apply_preconditioner(d, rr, ncols).reshape(ncols, -1)
                # complex64 both ways, the K slices summed in another order (5e-5: the twisted
                # strip solves, the default at bcr = 0, amplify it more than block Thomas)
                assert rel(zp, zl) < (5e-5 if bcr == 0 else 1e-5), (d, single)
                sw = sweep.Sweeper(A, k, n, N, d)
                for c in range(ncols):
                    assert rel(zp[c], sw.apply(r[c], not single)) < 2e-4, (d, c, single)
            # one launch per sweep besides the column tables, pack and unpack (graph replays count
            # their kernels); the phase-by-phase form launches every phase
            lp, ll = hp.stats()["kernel_launches"], hl.stats()["kernel_launches"]
            assert lp <= 4 * 4, lp
            assert ll > lp


def test_fp32_first_gram_schmidt_pass():
    """With complex64 sweeps the first Gram-Schmidt pass takes its inner products in FP32 and
    the FP64 second pass corrects them: the same iterations as both passes in FP64, the same
    solution to rounding, and the explicit residual on the implicit one (the Arnoldi relation
    stays FP64-accurate)."""
    k, n, N = 60.0, 128, 8
    P = solver.Problem(k, n, N)
    b = P.rhs(hh_inputs.centre_source())
    with hh.Handle(k, n, N, precision="fp32", gs_tensor=0) as h1, \
            hh.Handle(k, n, N, precision="fp32", gs_first_fp32=0, gs_tensor=0) as h0:
        x1, r1 = h1.solve(b, tol=1e-8)
        x0, r0 = h0.solve(b, tol=1e-8)
    assert r1.status == hh.HH_OK and r0.status == hh.HH_OK
    assert abs(r1.iterations - r0.iterations) <= 1
    assert rel(x1, x0) < 1e-6
    assert r1.rel_res_explicit < 2 * max(r1.rel_res_implicit, 1e-10)


@pytest.mark.parametrize("dirs", ["BT", "LR+BT", "LR+BT+RL", "LR+RL+BT+TB"])
@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_tensor_core_gram_schmidt(dirs, precision):
    """Gram-Schmidt against the basis as exact integer products of 7-bit slices on the tensor
    cores (hh_opts.gs_tensor = 1) against the FP64-pipe kernels: FP64-accurate inner products
    and updates give the same iterations, the same solution to rounding, and the explicit
    residual on the implicit one, for t = 1..4 new columns per iteration.  The two round
    differently (FP64 sums in another order; slices truncated at 2^-56 of a vector's largest
    entry), and the Krylov basis amplifies that: FP64 solutions agree to 1e-11, ten times
    inside the oracle parity bar."""
    k, n, N = 60.0, 128, 8
    P = solver.Problem(k, n, N)
    b = P.rhs(hh_inputs.centre_source())
    with hh.Handle(k, n, N, dirs, precision=precision) as h1, \
            hh.Handle(k, n, N, dirs, precision=precision, gs_tensor=0) as h0:
        x1, r1 = h1.solve(b, tol=1e-10)
        x0, r0 = h0.solve(b, tol=1e-10)
    assert r1.status == hh.HH_OK and r0.status == hh.HH_OK
    assert r1.iterations == r0.iterations
    assert rel(x1, x0) < (1e-11 if precision == "fp64" else 1e-9)
    assert r1.rel_res_explicit < 2 * max(r1.rel_res_implicit, 1e-12)


def test_tensor_core_gram_schmidt_long_basis():
    """More than 128 basis vectors (two tensor-memory rounds of the inner products, three
    exact-accumulation segments of the update) with single sweeps to a tight tolerance: the
    same iterations and solution as the FP64-pipe kernels."""
    k, n, N = 40.0, 64, 8
    P = solver.Problem(k, n, N)
    b = P.rhs(hh_inputs.centre_source())
    kw = dict(precision="fp64", single_sweep=1, maxit=60)
    with hh.Handle(k, n, N, "LR+RL+BT+TB", **kw) as h1, \
            hh.Handle(k, n, N, "LR+RL+BT+TB", gs_tensor=0, **kw) as h0:
        x1, r1 = h1.solve(b, tol=1e-13)
        x0, r0 = h0.solve(b, tol=1e-13)
    assert r0.iterations >= 33, r0.iterations  # 1 + 4 x 32 > 128 basis vectors
    assert abs(r1.iterations - r0.iterations) <= 1
    assert rel(x1, x0) < 1e-10
    assert r1.rel_res_explicit < 10 * max(r1.rel_res_implicit, 1e-13)


BF16_SWEEP_BAR = 3e-2


@pytest.mark.parametrize("k,n,N", [(20.0, 32, 4), (40.0, 256, 16), (30.0, 96, 3)])
@pytest.mark.parametrize("bcr", [0, 2])
def test_bf16_sweeps(k, n, N, bcr):
    """HH_PREC_BF16 (Section 5's lower-precision subsolves): the factors in bf16 and one bf16
    tensor-core product per K step with FP32 accumulation.  Every product rounds its factor
    entries and line values to 8 significant bits (relative 2^-9); the sweep stays within a few
    per cent of the oracle's (banded LU in FP64), for the double and single sweeps, 4 columns."""
    R = n // N
    if R % (1 << bcr):
        pytest.skip("depth needs R divisible by 2^d")
    A, *_ = fem.global_system(k, n)
    r = hh_inputs.random_vector(A.shape[0], 4, seed=60)
    rr = np.ascontiguousarray(r.ravel())
    for single in (0, 1):
        with hh.Handle(k, n, N, precision="bf16", bcr_depth=bcr, single_sweep=single) as h:
            for d in sweep.DIRECTIONS:
                z = h.apply_preconditioner(d, rr, 4).reshape(4, -1)
                sw = sweep.Sweeper(A, k, n, N, d)
                errs = [rel(z[c], sw.apply(r[c], not single)) for c in range(4)]
                assert max(errs) < BF16_SWEEP_BAR, (d, single, errs)
                assert max(errs) > 1e-5  # the products really are bf16


@pytest.mark.parametrize("k,n,N", [(60.0, 128, 8), (100.0, 256, 16)])
def test_bf16_solve_converges(k, n, N):
    """Flexible MPGMRES with bf16 sweeps reaches tol 1e-6 in explicit residual (the Krylov side is
    FP64), within a few iterations of the oracle's FP64 preconditioners, and the solution
    agrees with the oracle's to the tolerance's level."""
    P = solver.Problem(k, n, N)
    b = P.rhs(hh_inputs.centre_source())
    ref = P.solve(b, tol=1e-6)
    with hh.Handle(k, n, N, precision="bf16") as h:
        x, res = h.solve(b, tol=1e-6)
    assert res.status == hh.HH_OK
    assert res.rel_res_explicit < 1.5e-6
    assert res.iterations <= ref.iterations + 6, (res.iterations, ref.iterations)
    assert rel(x, ref.x) < 1e-4


def _gs_inputs(D, p, t, seed):
    """Basis columns of unit norm with a few large entries, new columns of very different
    scales (1, 1e-9, 1e7, and one with a single spike)."""
    rng = np.random.default_rng(seed)
    V = rng.standard_normal((p, D)) + 1j * rng.standard_normal((p, D))
    V[:, rng.integers(0, D, 5)] *= 40.0
    V /= np.linalg.norm(V, axis=1, keepdims=True)
    W = rng.standard_normal((t, D)) + 1j * rng.standard_normal((t, D))
    scales = [1.0, 1e-9, 1e7, 1.0][:t]
    W *= np.array(scales)[:, None]
    if t == 4:
        W[3] *= 1e-6
        W[3, D // 3] = 3.0 + 4.0j
    W += 0.3 * (V[:t].T @ np.eye(t)).T * np.array(scales)[:, None]  # a part inside the basis
    return np.ascontiguousarray(V), np.ascontiguousarray(W)


@pytest.mark.parametrize("gs_tensor", [1, 0])
@pytest.mark.parametrize("p,t", [(37, 4), (5, 1), (130, 3)])
def test_gram_schmidt_pass_fp64_bound(gs_tensor, p, t):
    """hh_gram_schmidt_pass against an 80-bit (long double) reference of H = V^H W and of
    W - V H (with the GPU's own H).

    FP64-pipe kernels: every inner product within 4u of sum |v||w| (u = 2^-53; the sums are
    blocked over threads and CTAs, far inside Higham's gamma_n), every updated entry within
    2 (p + 4) u of sum_a |v_a||h_ab| + |result| (the worst case of a p-term sum, doubled for
    the three-multiplication complex product).
    Tensor cores: the same terms plus the slice truncation, which is relative to each vector's
    largest entry (|dv| < 2^-55 max|v|, |dw| < 2^-55 max|w|, |dh_ab| < 2^-54 max_a |h_ab| m_a /
    m_a with m_a = max|v_a|): 2^-53 (max|v| |w|_1 + max|w| |v|_1) per inner product and
    2^-53 (sum_a m_a |h_ab| + max_a (m_a |h_ab|) sum_a |v_a| / m_a) per updated entry.  A
    typical-case check on top: every inner product within 1e-15 |v| |w| (the truncation errors
    have random signs; the worst case is sqrt(2 D) times larger)."""
    k, n, N = 30.0, 96, 4
    D = (n + 1) ** 2
    V, W = _gs_inputs(D, p, t, seed=11 + p)
    ld = np.longdouble
    Vr, Vi = V.real.astype(ld), V.imag.astype(ld)
    Wr, Wi = W.real.astype(ld), W.imag.astype(ld)
    Hr = Vr @ Wr.T + Vi @ Wi.T          # Re conj(v) w
    Hi = Vr @ Wi.T - Vi @ Wr.T          # Im conj(v) w
    aV, aW = np.abs(V), np.abs(W)
    with hh.Handle(k, n, N, gs_tensor=gs_tensor) as h:
        W1 = W.copy()
        H = h.gram_schmidt_pass(V.ravel(), p, W1.ravel(), t)
        W1 = W1.reshape(t, D)
    u = 2.0 ** -53
    mv, mw = aV.max(axis=1), aW.max(axis=1)
    bound_h = 4 * u * (aV @ aW.T)
    if gs_tensor:
        bound_h = bound_h + u * (np.outer(mv, aW.sum(axis=1)) + np.outer(aV.sum(axis=1), mw))
    err_h = np.abs(H - (Hr.astype(np.float64) + 1j * Hi.astype(np.float64)))
    assert np.all(err_h <= bound_h), float(np.max(err_h / bound_h))
    if gs_tensor:
        nv = np.linalg.norm(V, axis=1)[:, None] * np.linalg.norm(W, axis=1)[None, :]
        assert np.all(err_h <= 1e-15 * nv), float(np.max(err_h / nv))
    Hg_r, Hg_i = H.real.astype(ld), H.imag.astype(ld)
    Ur = Wr - (Vr.T @ Hg_r - Vi.T @ Hg_i).T
    Ui = Wi - (Vr.T @ Hg_i + Vi.T @ Hg_r).T
    err_w = np.abs(W1 - (Ur.astype(np.float64) + 1j * Ui.astype(np.float64)))
    aH = np.abs(H)
    bound_w = (4 if gs_tensor else 2 * (p + 4)) * u * ((aV.T @ aH).T + np.abs(W1))
    if gs_tensor:
        mh = (mv[:, None] * aH).max(axis=0)                       # max_a m_a |h_ab|, per b
        bound_w = bound_w + u * ((mv @ aH)[:, None] + mh[:, None] * (aV / mv[:, None]).sum(axis=0)[None, :])
    assert np.all(err_w <= bound_w), float(np.max(err_w / bound_w))
