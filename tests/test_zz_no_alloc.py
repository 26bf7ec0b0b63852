"""hh_apply_preconditioner_noalloc: the preconditioner apply for callers that cannot
allocate device memory during a call (fixed device-memory budgets, host frameworks that own
the device allocator, latency-critical paths that must avoid cudaMalloc / cudaFree).

The entry point must give the same result as hh_apply_preconditioner, which allocates its
own workspaces, and keep doing so on repeated calls, since every call reuses one fixed
scratch array that still holds the previous call's data.  This file is collected last so
that a run stopping at the first failure has already run every other test.
"""
import ctypes

import numpy as np
import pytest

import hh_inputs
import paper_2408_11929_gb300 as hh

pytestmark = pytest.mark.gpu

# same tolerances as the allocating entry point's parity tests (FP64 / FP32 sweeps)
TOL = {"fp64": 1e-10, "fp32": 2e-4}


@pytest.fixture(scope="module", autouse=True)
def built():
    import __graft_entry__
    __graft_entry__.build()


def rel(a, b):
    a = a.cpu().numpy().ravel()
    b = b.cpu().numpy().ravel()
    return np.linalg.norm(a - b) / np.linalg.norm(b)


def noalloc(h, d, ncols, r, torch):
    z = torch.full_like(r, complex(np.nan, np.nan))
    st = h.lib.hh_apply_preconditioner_noalloc(h.h, hh.DIR_BITS[d], ncols, ctypes.c_void_p(r.data_ptr()),
                                               ctypes.c_void_p(z.data_ptr()))
    torch.cuda.synchronize()
    assert st == hh.HH_OK, h.lib.hh_last_error()
    return z


# complex64 with an even column count runs the tensor-core step (tensor maps over the fixed
# array, split-K slices in what is left of it); an odd count and complex128 the CUDA-core one
@pytest.mark.parametrize("precision,ncols", [("fp64", 3), ("fp32", 2), ("fp32", 3), ("fp32", 4)])
def test_noalloc_matches_allocating_entry_point(precision, ncols):
    torch = pytest.importorskip("torch")
    k, n, N = 30.0, 64, 4
    dofs = (n + 1) ** 2
    r = torch.from_numpy(np.ascontiguousarray(hh_inputs.random_vector(dofs, ncols, seed=5).ravel())).cuda()
    with hh.Handle(k, n, N, precision=precision) as h:
        for d in ("LR", "TB", "BT", "RL"):
            z_ref = h.apply_preconditioner(d, r, ncols)
            for call in range(2):  # two calls in a row reuse the scratch left by the previous one
                z = noalloc(h, d, ncols, r, torch)
                assert rel(z, z_ref) <= TOL[precision], (d, call)


def test_noalloc_before_any_allocating_call():
    """The first calls on a fresh handle, before the allocating entry point has run (so no
    tensor-core candidate has been tuned for the column count), agree with a later
    allocating call."""
    torch = pytest.importorskip("torch")
    k, n, N, ncols = 30.0, 64, 4, 4
    dofs = (n + 1) ** 2
    r = torch.from_numpy(np.ascontiguousarray(hh_inputs.random_vector(dofs, ncols, seed=7).ravel())).cuda()
    with hh.Handle(k, n, N, precision="fp32") as h:
        z = [noalloc(h, "BT", ncols, r, torch) for _ in range(2)]
        z_ref = h.apply_preconditioner("BT", r, ncols)
        for call in range(2):
            assert rel(z[call], z_ref) <= TOL["fp32"], call


def test_noalloc_rejects_what_it_cannot_serve():
    torch = pytest.importorskip("torch")
    k, n, N = 30.0, 64, 4
    dofs = (n + 1) ** 2
    with hh.Handle(k, n, N) as h:
        lib = h.lib
        # host buffers would need a staging copy on the device
        rh = np.zeros(dofs, dtype=np.complex128)
        zh = np.zeros(dofs, dtype=np.complex128)
        st = lib.hh_apply_preconditioner_noalloc(h.h, hh.HH_DIR_LR, 1, ctypes.c_void_p(rh.ctypes.data),
                                                 ctypes.c_void_p(zh.ctypes.data))
        assert st == hh.HH_EINVAL
        # more columns than the fixed scratch can hold
        big = 2000
        r = torch.zeros(dofs * big, dtype=torch.complex128, device="cuda")
        z = torch.zeros_like(r)
        st = lib.hh_apply_preconditioner_noalloc(h.h, hh.HH_DIR_LR, big, ctypes.c_void_p(r.data_ptr()),
                                                 ctypes.c_void_p(z.data_ptr()))
        assert st == hh.HH_EINVAL
        assert b"scratch" in lib.hh_last_error()
        # the handle still works after the rejections
        rs = torch.from_numpy(np.ascontiguousarray(hh_inputs.random_vector(dofs, 1, seed=6).ravel())).cuda()
        zs = torch.zeros_like(rs)
        st = lib.hh_apply_preconditioner_noalloc(h.h, hh.HH_DIR_BT, 1, ctypes.c_void_p(rs.data_ptr()),
                                                 ctypes.c_void_p(zs.data_ptr()))
        assert st == hh.HH_OK
        assert rel(zs, h.apply_preconditioner("BT", rs)) <= TOL["fp64"]
