"""Whole-method driver: assemble, build the directional sweeps, run MPGMRES.

Direction strings use the vocabulary of Section 4: LR, RL, BT, TB name the direction of
the FORWARD pass; a double sweep (LRL, RLR, BTB, TBT) is the default, ``double=False``
gives the single (forward-only) sweeps.  "LR+BT" is the paper's LRL+BTB combination.
"""
from __future__ import annotations

import numpy as np

from . import fem, mpgmres, sweep


def parse_dirs(dirs: str) -> list[str]:
    out = [d.strip().upper() for d in dirs.split("+") if d.strip()]
    for d in out:
        if d not in sweep.DIRECTIONS:
            raise ValueError(f"unknown direction {d}")
    return out


class Problem:
    """Assembled operator and the t preconditioners for one (k, n, N, dirs)."""

    def __init__(self, k: float, n: int, N: int, dirs: str = "LR+RL+BT+TB", double: bool = True,
                 cache: bool = True):
        self.k, self.n, self.N = k, n, N
        self.dirs = parse_dirs(dirs)
        self.A, self.K, self.M, self.MG = fem.global_system(k, n)
        self.cache = sweep.FactorCache(cache)
        self.sweepers = [sweep.Sweeper(self.A, k, n, N, d, self.cache) for d in self.dirs]
        self.double = double
        self.precs = [(lambda r, sw=sw: sw.apply(r, double)) for sw in self.sweepers]

    def rhs(self, sources) -> np.ndarray:
        return fem.load_vector(self.n, self.M, self.MG, fem.gaussian_source(self.n, sources))

    def solve(self, b: np.ndarray, tol: float, maxit: int = 200, scheme: str = "auto",
              **kw) -> mpgmres.Result:
        return mpgmres.solve(self.A, self.precs, b, tol=tol, maxit=maxit, scheme=scheme, **kw)
