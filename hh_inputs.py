"""Seeded synthetic inputs shared by the oracle, the tests and the benchmark.

This module only draws random numbers and describes workloads; it contains none of
the method's arithmetic (no assembly, no source evaluation, no solver step).  Each
side (the CPU oracle and the CUDA library) turns these parameters into a load vector
on its own.

Source model (the paper's benchmark is a point-like Gaussian source in the unit
square, Section 4): every right-hand side is a list of Gaussian bumps
    f(x, y) = amp * exp(-((x - x0)^2 + (y - y0)^2) / (2 sigma^2))
described by rows (x0, y0, sigma, amp.real, amp.imag).
"""
from __future__ import annotations

from dataclasses import dataclass, field
from typing import List, Optional

import numpy as np

SIGMA = 0.05


@dataclass
class Workload:
    """One solve configuration: wave number, grid, strips, directions, sources."""

    name: str
    k: float
    n: int                 # cells per side; nodes per side m = n + 1
    strips: int            # N strips of R = n / N node lines each (last one R + 1)
    dirs: str              # subset of "LR,RL,BT,TB" joined by '+'
    nrhs: int
    tol: float
    precision: str         # "fp64" or "fp32" (precision of the strip factors and sweeps)
    sources: List[np.ndarray] = field(default_factory=list)  # per RHS: (nsrc, 5) float64

    @property
    def m(self) -> int:
        return self.n + 1

    @property
    def dofs(self) -> int:
        return (self.n + 1) ** 2


def centre_source(amp: complex = 1.0) -> np.ndarray:
    return np.array([[0.5, 0.5, SIGMA, float(np.real(amp)), float(np.imag(amp))]], dtype=np.float64)


def random_sources(nrhs: int, seed: int = 0, complex_amp: bool = False) -> List[np.ndarray]:
    """nrhs single-Gaussian sources at uniform locations in [0.1, 0.9]^2.

    Amplitude 1, or complex normal (N(0,1) + i N(0,1)) / sqrt(2) when complex_amp.
    """
    rng = np.random.default_rng(seed)
    xy = rng.uniform(0.1, 0.9, size=(nrhs, 2))
    if complex_amp:
        a = (rng.standard_normal(nrhs) + 1j * rng.standard_normal(nrhs)) / np.sqrt(2.0)
    else:
        a = np.ones(nrhs, dtype=np.complex128)
    return [np.array([[xy[r, 0], xy[r, 1], SIGMA, a[r].real, a[r].imag]]) for r in range(nrhs)]


def random_vector(dofs: int, ncols: int = 1, seed: int = 0) -> np.ndarray:
    """Complex normal test vectors, shape (ncols, dofs), complex128."""
    rng = np.random.default_rng(seed)
    return (rng.standard_normal((ncols, dofs)) + 1j * rng.standard_normal((ncols, dofs))) / np.sqrt(2.0)


def workload(name: str) -> Workload:
    """The named synthetic workloads (sizes and source recipes)."""
    if name == "k20_n32":          # plain method, FP64, small
        return Workload(name, 20.0, 32, 4, "LR+RL+BT+TB", 1, 1e-8, "fp64", [centre_source()])
    if name == "k100_n256":        # FP64 path, 8 RHS at random interior points
        return Workload(name, 100.0, 256, 16, "LR+RL+BT+TB", 8, 1e-8, "fp64", random_sources(8, 0))
    if name == "k400_n1024":       # precision config: FP32 sweeps, FP64 outer
        return Workload(name, 400.0, 1024, 32, "LR+RL+BT+TB", 1, 1e-6, "fp32", [centre_source()])
    if name == "k200_n512_b64":    # batching config: 64 RHS, complex normal amplitudes
        return Workload(name, 200.0, 512, 16, "LR+RL+BT+TB", 64, 1e-6, "fp32",
                        random_sources(64, 0, complex_amp=True))
    raise KeyError(name)


def serving_stream(nreq: int = 500, seed: int = 0, rate_hz: Optional[float] = None):
    """Mixed-k request stream: k integer uniform in [50, 400], n = ceil(2.5 k / 32) * 32,
    strips of 32 node lines, one Gaussian source each, Poisson arrival times."""
    rng = np.random.default_rng(seed)
    ks = rng.integers(50, 401, size=nreq).astype(np.float64)
    ns = (np.ceil(2.5 * ks / 32.0) * 32).astype(int)
    xy = rng.uniform(0.1, 0.9, size=(nreq, 2))
    gaps = rng.exponential(1.0, size=nreq)
    reqs = []
    for r in range(nreq):
        reqs.append(dict(k=float(ks[r]), n=int(ns[r]), strips=int(ns[r] // 32),
                         sources=np.array([[xy[r, 0], xy[r, 1], SIGMA, 1.0, 0.0]]),
                         gap=float(gaps[r])))
    if rate_hz is not None:
        t = 0.0
        for q in reqs:
            t += q["gap"] / rate_hz
            q["t_arrive"] = t
    return reqs
