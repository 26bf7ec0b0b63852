"""Serving (hh_server_*): requests for several problems (k, n) behind one submit / poll
interface, with a device-resident factor cache admitted by memory.  Every result must equal
the same problem solved on its own handle (same iteration count; FP64 solutions within
1e-10 relative), whether it came from a cached handle, a fresh one, or one rebuilt after an
eviction."""
import time

import numpy as np
import pytest

import hh_inputs
import paper_2408_11929_gb300 as hh

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    import __graft_entry__
    __graft_entry__.build()


def rel(a, b):
    return np.linalg.norm(np.ravel(a) - np.ravel(b)) / np.linalg.norm(np.ravel(b))


def wait_all(srv, tickets, timeout=120):
    done = {}
    t0 = time.time()
    while len(done) < len(tickets) and time.time() - t0 < timeout:
        for t in tickets:
            if t not in done:
                st, res = srv.poll(t)
                if st != hh.HH_EPENDING:
                    done[t] = (st, res)
        time.sleep(0.001)
    assert len(done) == len(tickets)
    return done


def alone(k, n, strips, src, tol):
    with hh.Handle(k, n, strips) as h:
        b = h.assemble_rhs(src)
        return h.solve(b, tol=tol)


PROBLEMS = [(20.0, 32, 4), (30.0, 64, 2), (20.0, 32, 4), (30.0, 64, 2), (20.0, 32, 4)]


def test_server_matches_dedicated_handles():
    srcs = hh_inputs.random_sources(len(PROBLEMS), seed=31)
    with hh.Server(serve_slots=2) as srv:
        xs = [np.zeros((n + 1) ** 2, dtype=np.complex128) for _, n, _ in PROBLEMS]
        tickets = [srv.submit(k, n, N, s, x, tol=1e-8) for (k, n, N), s, x in zip(PROBLEMS, srcs, xs)]
        done = wait_all(srv, tickets)
        st = srv.stats()
    assert st["setups"] == 2 and st["cache_hits"] == 3 and st["completed"] == 5
    for (k, n, N), s, x, t in zip(PROBLEMS, srcs, xs, tickets):
        xa, ra = alone(k, n, N, s, 1e-8)
        status, res = done[t]
        assert status == hh.HH_OK and res.iterations == ra.iterations
        assert res.rel_res_explicit < 1e-8
        assert res.t_solve_ms > 0
        assert rel(x, xa) < 1e-10


def test_server_evicts_to_stay_within_budget():
    """A budget that holds one of two equally sized problems: alternating requests evict
    and rebuild, and every result is still the dedicated-handle result."""
    src = hh_inputs.random_sources(4, seed=32)
    with hh.Server(serve_slots=1) as probe:
        x = np.zeros(33 * 33, dtype=np.complex128)
        wait_all(probe, [probe.submit(20.0, 32, 4, src[0], x, tol=1e-8)])
        one = probe.stats()["bytes_reserved"]
    probs = [(20.0, 32, 4), (25.0, 32, 4), (20.0, 32, 4), (25.0, 32, 4)]
    with hh.Server(mem_budget=int(one * 1.5), serve_slots=1) as srv:
        xs = [np.zeros(33 * 33, dtype=np.complex128) for _ in probs]
        tickets = []
        for (k, n, N), s, x in zip(probs, src, xs):
            tickets.append(srv.submit(k, n, N, s, x, tol=1e-8))
            wait_all(srv, tickets[-1:])  # one at a time, so the other problem's handle is idle
        st = srv.stats()
    assert st["evictions"] >= 3 and st["handles"] == 1 and st["setups"] == 4
    for (k, n, N), s, x in zip(probs, src, xs):
        xa, _ = alone(k, n, N, s, 1e-8)
        assert rel(x, xa) < 1e-10
