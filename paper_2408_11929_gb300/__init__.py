"""Python binding of libhh, the GB300 multipreconditioned directional-sweep Helmholtz solver.

Thin ctypes marshalling over the C ABI declared in include/hh.h: every computation runs
in the library's CUDA kernels.  Vectors are complex128, (n+1)^2 entries per column in
node order g = j (n+1) + i; they may be numpy arrays (host memory, copied by the library)
or CUDA torch tensors (device memory, used in place).  There is no CPU fallback: loading
fails loudly when the compiled library is missing.
"""
from __future__ import annotations

import ctypes
import os
from typing import Optional, Sequence

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libhh.so")

HH_OK, HH_EINVAL, HH_ENOMEM, HH_ENOCONV, HH_EBREAKDOWN, HH_ENAN, HH_ETIMEOUT, HH_EPENDING, HH_ECUDA = range(9)
STATUS_NAMES = ["OK", "EINVAL", "ENOMEM", "ENOCONV", "EBREAKDOWN", "ENAN", "ETIMEOUT", "EPENDING", "ECUDA"]
HH_DIR_LR, HH_DIR_RL, HH_DIR_BT, HH_DIR_TB = 1, 2, 4, 8
DIR_BITS = {"LR": HH_DIR_LR, "RL": HH_DIR_RL, "BT": HH_DIR_BT, "TB": HH_DIR_TB}
HH_PREC_FP64, HH_PREC_FP32, HH_PREC_BF16 = 0, 1, 2
HH_SCHEME_AUTO, HH_SCHEME_CROSS, HH_SCHEME_SUM = 0, 1, 2
HH_DISC_P1, HH_DISC_FD = 0, 1


class hh_opts(ctypes.Structure):
    _fields_ = [("precision", ctypes.c_int), ("scheme", ctypes.c_int), ("single_sweep", ctypes.c_int),
                ("maxit", ctypes.c_int), ("deflate_eta", ctypes.c_double), ("bcr_depth", ctypes.c_int),
                ("timeout_cycles", ctypes.c_int64), ("stream", ctypes.c_void_p), ("use_graph", ctypes.c_int),
                ("profile", ctypes.c_int), ("gs_passes", ctypes.c_int), ("serve_slots", ctypes.c_int),
                ("tensor_cores", ctypes.c_int), ("autotune", ctypes.c_int), ("fuse_chains", ctypes.c_int),
                ("overlap_steps", ctypes.c_int), ("interface_form", ctypes.c_int),
                ("persistent", ctypes.c_int), ("gs_first_fp32", ctypes.c_int),
                ("discretization", ctypes.c_int), ("group_wide_tiles", ctypes.c_int), ("gs_tensor", ctypes.c_int),
                ("twisted", ctypes.c_int)]


class hh_result(ctypes.Structure):
    _fields_ = [("iterations", ctypes.c_int), ("rel_res_implicit", ctypes.c_double),
                ("rel_res_explicit", ctypes.c_double), ("t_setup_ms", ctypes.c_double),
                ("t_solve_ms", ctypes.c_double), ("status", ctypes.c_int)]

    def as_dict(self) -> dict:
        return {f: getattr(self, f) for f, _ in self._fields_}


class hh_stats(ctypes.Structure):
    _fields_ = [("sweep_launches", ctypes.c_int64), ("sweep_ms", ctypes.c_double), ("sweep_bytes", ctypes.c_double),
                ("spmv_launches", ctypes.c_int64), ("spmv_ms", ctypes.c_double), ("spmv_bytes", ctypes.c_double),
                ("gs_launches", ctypes.c_int64), ("gs_ms", ctypes.c_double), ("gs_bytes", ctypes.c_double),
                ("setup_launches", ctypes.c_int64), ("setup_ms", ctypes.c_double), ("setup_flops", ctypes.c_double),
                ("kernel_launches", ctypes.c_int64), ("factor_bytes", ctypes.c_int64), ("factor_blocks", ctypes.c_int),
                ("m", ctypes.c_int), ("ldf", ctypes.c_int), ("columns", ctypes.c_int), ("sweep_steps", ctypes.c_int64),
                ("gemm_launches", ctypes.c_int64), ("gemm_ms", ctypes.c_double), ("gemm_flops", ctypes.c_double),
                ("tensor_cores", ctypes.c_int), ("gsdot_launches", ctypes.c_int64), ("gsdot_ms", ctypes.c_double),
                ("gsdot_flops", ctypes.c_double), ("gs_flops", ctypes.c_double), ("wide_steps", ctypes.c_int64),
                ("ns_blocks", ctypes.c_int), ("ns_iterations", ctypes.c_int), ("tc_bnc", ctypes.c_int),
                ("tc_nsplit", ctypes.c_int), ("tc_cluster", ctypes.c_int), ("tc_us", ctypes.c_double), ("iterations_total", ctypes.c_int64),
                ("step_graphs", ctypes.c_int), ("step_graph_fallback", ctypes.c_int), ("bcr_depth", ctypes.c_int),
                ("gsdot_bytes", ctypes.c_double), ("twisted", ctypes.c_int)]

    def as_dict(self) -> dict:
        return {f: getattr(self, f) for f, _ in self._fields_}


class hh_server_stats(ctypes.Structure):
    _fields_ = [("handles", ctypes.c_int64), ("bytes_reserved", ctypes.c_int64), ("budget", ctypes.c_int64),
                ("setups", ctypes.c_int64), ("cache_hits", ctypes.c_int64), ("evictions", ctypes.c_int64),
                ("completed", ctypes.c_int64), ("queued", ctypes.c_int64), ("running", ctypes.c_int64),
                ("setup_ms", ctypes.c_double)]

    def as_dict(self) -> dict:
        return {f: getattr(self, f) for f, _ in self._fields_}


EXPORTS = ["hh_default_opts", "hh_setup", "hh_solve", "hh_solve_batch", "hh_submit", "hh_poll", "hh_assemble_rhs",
           "hh_apply_operator", "hh_apply_preconditioner", "hh_apply_preconditioner_noalloc", "hh_gram_schmidt_pass",
           "hh_get_factor",
           "hh_get_stats", "hh_reset_stats", "hh_destroy", "hh_last_error", "hh_server_create", "hh_server_submit",
           "hh_server_poll", "hh_server_get_stats", "hh_server_destroy"]

_lib = None


def load(path: str = LIB_PATH) -> ctypes.CDLL:
    """Load libhh.so (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError(f"libhh.so is missing at {path}; run __graft_entry__.build() first")
    L = ctypes.CDLL(path)
    vp, i, d, u32 = ctypes.c_void_p, ctypes.c_int, ctypes.c_double, ctypes.c_uint32
    L.hh_default_opts.argtypes = [ctypes.POINTER(hh_opts)]
    L.hh_default_opts.restype = None
    L.hh_setup.argtypes = [d, i, i, u32, ctypes.POINTER(hh_opts), ctypes.POINTER(vp)]
    L.hh_solve.argtypes = [vp, vp, vp, d, ctypes.POINTER(hh_result)]
    L.hh_solve_batch.argtypes = [vp, i, vp, vp, d, ctypes.POINTER(hh_result)]
    L.hh_submit.argtypes = [vp, vp, vp, d, ctypes.POINTER(ctypes.c_uint64)]
    L.hh_poll.argtypes = [ctypes.c_uint64, ctypes.POINTER(hh_result)]
    L.hh_assemble_rhs.argtypes = [vp, i, vp, vp]
    L.hh_apply_operator.argtypes = [vp, i, vp, vp]
    L.hh_apply_preconditioner.argtypes = [vp, u32, i, vp, vp]
    L.hh_apply_preconditioner_noalloc.argtypes = [vp, u32, i, vp, vp]
    L.hh_gram_schmidt_pass.argtypes = [vp, i, vp, i, vp, vp]
    L.hh_get_factor.argtypes = [vp, i, vp]
    L.hh_get_stats.argtypes = [vp, ctypes.POINTER(hh_stats)]
    L.hh_reset_stats.argtypes = [vp]
    L.hh_reset_stats.restype = None
    L.hh_destroy.argtypes = [vp]
    L.hh_destroy.restype = None
    L.hh_last_error.argtypes = []
    L.hh_last_error.restype = ctypes.c_char_p
    L.hh_server_create.argtypes = [ctypes.POINTER(hh_opts), ctypes.c_size_t, ctypes.POINTER(vp)]
    L.hh_server_submit.argtypes = [vp, d, i, i, u32, i, vp, vp, d, ctypes.POINTER(ctypes.c_uint64)]
    L.hh_server_poll.argtypes = [vp, ctypes.c_uint64, ctypes.POINTER(hh_result)]
    L.hh_server_get_stats.argtypes = [vp, ctypes.POINTER(hh_server_stats)]
    L.hh_server_destroy.argtypes = [vp]
    L.hh_server_destroy.restype = None
    for name in EXPORTS:
        if name not in ("hh_default_opts", "hh_reset_stats", "hh_destroy", "hh_last_error", "hh_server_destroy"):
            getattr(L, name).restype = ctypes.c_int
    _lib = L
    return L


class HHError(RuntimeError):
    def __init__(self, status: int, where: str):
        msg = load().hh_last_error().decode(errors="replace")
        super().__init__(f"{where}: {STATUS_NAMES[status] if 0 <= status < 9 else status}: {msg}")
        self.status = status


def dirs_mask(dirs) -> int:
    if isinstance(dirs, int):
        return dirs
    return sum(DIR_BITS[d.strip().upper()] for d in dirs.split("+") if d.strip())


def default_opts(**kw) -> hh_opts:
    o = hh_opts()
    load().hh_default_opts(ctypes.byref(o))
    for k, v in kw.items():
        if k == "precision" and isinstance(v, str):
            v = (HH_PREC_FP32 if v.lower() in ("fp32", "c64", "float")
                 else HH_PREC_BF16 if v.lower() == "bf16" else HH_PREC_FP64)
        setattr(o, k, v)
    return o


def _ptr(a) -> int:
    """Raw pointer of a numpy array (host) or a torch tensor (device or host)."""
    if isinstance(a, np.ndarray):
        if a.dtype != np.complex128 or not a.flags.c_contiguous:
            raise TypeError("numpy arrays must be C-contiguous complex128")
        return a.ctypes.data
    dt = str(getattr(a, "dtype", ""))
    if dt != "torch.complex128" or not a.is_contiguous():
        raise TypeError("torch tensors must be contiguous complex128")
    return a.data_ptr()


def _empty_like(a, n: int):
    if isinstance(a, np.ndarray):
        return np.zeros(n, dtype=np.complex128)
    import torch
    return torch.zeros(n, dtype=torch.complex128, device=a.device)


class Handle:
    """hh_setup ... hh_destroy around one (k, n, strips, dirs) problem."""

    def __init__(self, k: float, n: int, strips: int, dirs="LR+RL+BT+TB", **opts):
        self.lib = load()
        self.k, self.n, self.strips = float(k), int(n), int(strips)
        self.m = self.n + 1
        self.dofs = self.m * self.m
        self.dirs = dirs_mask(dirs)
        self.opts = default_opts(**opts)
        h = ctypes.c_void_p()
        st = self.lib.hh_setup(self.k, self.n, self.strips, self.dirs, ctypes.byref(self.opts), ctypes.byref(h))
        if st != HH_OK:
            raise HHError(st, "hh_setup")
        self.h = h

    def close(self):
        if getattr(self, "h", None):
            self.lib.hh_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def _check(self, st: int, where: str, ok=(HH_OK,)):
        if st not in ok:
            raise HHError(st, where)
        return st

    def solve(self, rhs, x=None, tol: float = 1e-8, raise_on=(HH_EINVAL, HH_ENOMEM, HH_ECUDA, HH_ETIMEOUT)):
        """Returns (x, hh_result)."""
        x = _empty_like(rhs, self.dofs) if x is None else x
        res = hh_result()
        st = self.lib.hh_solve(self.h, _ptr(rhs), _ptr(x), float(tol), ctypes.byref(res))
        if st in raise_on:
            raise HHError(st, "hh_solve")
        return x, res

    def solve_batch(self, rhs, nrhs: int, x=None, tol: float = 1e-8,
                    raise_on=(HH_EINVAL, HH_ENOMEM, HH_ECUDA, HH_ETIMEOUT)):
        """rhs, x: nrhs columns stored one after the other.  Returns (x, [hh_result])."""
        x = _empty_like(rhs, self.dofs * nrhs) if x is None else x
        res = (hh_result * nrhs)()
        st = self.lib.hh_solve_batch(self.h, int(nrhs), _ptr(rhs), _ptr(x), float(tol), res)
        if st in raise_on:
            raise HHError(st, "hh_solve_batch")
        return x, list(res)

    def submit(self, rhs, x, tol: float = 1e-8) -> int:
        t = ctypes.c_uint64()
        self._check(self.lib.hh_submit(self.h, _ptr(rhs), _ptr(x), float(tol), ctypes.byref(t)), "hh_submit")
        return t.value

    def poll(self, ticket: int):
        """(status, hh_result or None); HH_EPENDING while running."""
        res = hh_result()
        st = self.lib.hh_poll(ctypes.c_uint64(ticket), ctypes.byref(res))
        return st, (None if st == HH_EPENDING else res)

    def assemble_rhs(self, sources, out=None):
        src = np.ascontiguousarray(np.atleast_2d(np.asarray(sources, dtype=np.float64)))
        out = np.zeros(self.dofs, dtype=np.complex128) if out is None else out
        self._check(self.lib.hh_assemble_rhs(self.h, src.shape[0], src.ctypes.data, _ptr(out)), "hh_assemble_rhs")
        return out

    def apply_operator(self, x, ncols: int = 1, y=None):
        y = _empty_like(x, self.dofs * ncols) if y is None else y
        self._check(self.lib.hh_apply_operator(self.h, int(ncols), _ptr(x), _ptr(y)), "hh_apply_operator")
        return y

    def apply_preconditioner(self, direction: str, r, ncols: int = 1, z=None):
        z = _empty_like(r, self.dofs * ncols) if z is None else z
        st = self.lib.hh_apply_preconditioner(self.h, DIR_BITS[direction], int(ncols), _ptr(r), _ptr(z))
        self._check(st, "hh_apply_preconditioner")
        return z

    def apply_preconditioner_noalloc(self, direction: str, r, z, ncols: int = 1) -> int:
        """hh_apply_preconditioner_noalloc: r, z device tensors; the library allocates nothing.
        Returns the status (HH_OK, or HH_EINVAL for host buffers / a request above the fixed
        scratch size)."""
        return self.lib.hh_apply_preconditioner_noalloc(self.h, DIR_BITS[direction], int(ncols), _ptr(r), _ptr(z))

    def gram_schmidt_pass(self, V, p: int, W, t: int) -> np.ndarray:
        """hh_gram_schmidt_pass: H = V^H W (returned, p x t complex128) and W <- W - V H in place
        (V: p columns, W: t columns, numpy arrays or device tensors)."""
        H = np.zeros(p * t, dtype=np.complex128)
        st = self.lib.hh_gram_schmidt_pass(self.h, int(p), _ptr(V), int(t), _ptr(W), H.ctypes.data)
        self._check(st, "hh_gram_schmidt_pass")
        return H.reshape(p, t)

    def get_factor(self, j: int) -> np.ndarray:
        out = np.zeros(self.m * self.m, dtype=np.complex128)
        self._check(self.lib.hh_get_factor(self.h, int(j), out.ctypes.data), "hh_get_factor")
        return out.reshape(self.m, self.m)

    def stats(self) -> dict:
        s = hh_stats()
        self._check(self.lib.hh_get_stats(self.h, ctypes.byref(s)), "hh_get_stats")
        return s.as_dict()

    def reset_stats(self):
        self.lib.hh_reset_stats(self.h)


class Server:
    """hh_server_create ... hh_server_destroy: solves of many problems (k, n) behind one
    submit / poll interface, with a device-resident factor cache admitted by memory."""

    def __init__(self, mem_budget: int = 0, **opts):
        self.lib = load()
        self.opts = default_opts(**opts)
        s = ctypes.c_void_p()
        st = self.lib.hh_server_create(ctypes.byref(self.opts), int(mem_budget), ctypes.byref(s))
        if st != HH_OK:
            raise HHError(st, "hh_server_create")
        self.s = s

    def submit(self, k: float, n: int, strips: int, sources, x, tol: float = 1e-6, dirs="LR+RL+BT+TB") -> int:
        src = np.ascontiguousarray(np.atleast_2d(np.asarray(sources, dtype=np.float64)))
        t = ctypes.c_uint64()
        st = self.lib.hh_server_submit(self.s, float(k), int(n), int(strips), dirs_mask(dirs), src.shape[0],
                                       src.ctypes.data, _ptr(x), float(tol), ctypes.byref(t))
        if st != HH_OK:
            raise HHError(st, "hh_server_submit")
        return t.value

    def poll(self, ticket: int):
        """(status, hh_result or None); HH_EPENDING while queued or running."""
        res = hh_result()
        st = self.lib.hh_server_poll(self.s, ctypes.c_uint64(ticket), ctypes.byref(res))
        return st, (None if st == HH_EPENDING else res)

    def stats(self) -> dict:
        st = hh_server_stats()
        if self.lib.hh_server_get_stats(self.s, ctypes.byref(st)) != HH_OK:
            raise HHError(HH_EINVAL, "hh_server_get_stats")
        return st.as_dict()

    def close(self):
        if getattr(self, "s", None):
            self.lib.hh_server_destroy(self.s)
            self.s = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()
