"""Selective flexible multipreconditioned GMRES (Section 3; selection rules of Section 4).

Right preconditioning, x0 = 0.  With t preconditioners, iteration k adds up to t search
directions Z_k = [M_i^{-1} s_i] and minimises ||b - A x|| over x in span(Z_1, ..., Z_k)
(Section 3: selective MPGMRES adds t vectors per iteration; flexible because every
preconditioner may be applied to a different vector and the Z vectors are stored).

One iteration:
  1. W = A Z_k.
  2. Block classical Gram-Schmidt against the current basis V, done twice (CGS2); the
     projection coefficients of both passes are summed into the new Hessenberg columns.
  3. The t columns of W are then orthonormalised one after the other, in preconditioner
     order, each by classical Gram-Schmidt against the new vectors already accepted in this
     iteration (again twice), giving a real positive diagonal r_jj.  Column j is DEFLATED (its Z column dropped)
     when r_jj == 0, or when another column of this block has been accepted already and
     r_jj <= eta * ||A z_j||, the norm of the new column before any Gram-Schmidt: the part of
     A z_j outside the span of the basis and of the block's accepted vectors is then below
     eta of its size, so the direction duplicates one already taken.  The first accepted
     column of a block is kept whenever r_jj > 0: when A z lies in the span of the basis
     (one strip, where the sweep is A^{-1}) it completes the least-squares problem (a lucky
     breakdown) even though its new basis vector is rounding noise.  (Section 3 gives no
     threshold.  Measuring r_jj against the norm left after step 2 instead keeps a direction
     that coincides with another new one to 1e-13 whenever step 2 already removed most of
     both: the triangular factor becomes ill-conditioned and x = Z y loses digits.)
  4. The Hessenberg matrix stays scalar upper Hessenberg; the previous complex Givens
     rotations are applied to each new column and one new rotation zeroes its
     sub-diagonal entry.  The residual estimate is |g_last|.
  5. Convergence is tested once per iteration, after all its columns:  rho / beta <= tol.
  6. Next sources (Section 4): one preconditioner -> the new basis vector; two -> each
     preconditioner is applied to the new basis vector that came from the OTHER
     preconditioner ("cross"); more than two -> all are applied to the normalised sum of
     the new basis vectors ("sum").  If a column was deflated its surviving partner is
     used.
At the end y solves the rotated triangular system, x = Z y, and the explicit relative
residual ||b - A x|| / ||b|| is reported.

``single_pass=True`` replaces the two Gram-Schmidt passes by one and counts inner
products, for the cost statement of Section 3: (k - 1/2) t^2 + (3/2) t at iteration k.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

ETA = 1e-10


@dataclass
class Result:
    x: np.ndarray
    iterations: int
    converged: bool
    status: str                      # "ok", "noconv", "breakdown"
    rel_res_implicit: float
    rel_res_explicit: float
    history: list = field(default_factory=list)   # rho_k / beta after every iteration
    inner_products: list = field(default_factory=list)  # per iteration (counted GS products)
    V: np.ndarray | None = None
    Z: np.ndarray | None = None
    H: np.ndarray | None = None      # unrotated (nV x nZ) Hessenberg matrix


def _givens(a: complex, b: complex):
    """c real, s complex with [[c, s], [-conj(s), c]] @ [a, b] = [r, 0]."""
    if b == 0:
        return 1.0, 0.0 + 0.0j
    if a == 0:
        return 0.0, np.conj(b) / abs(b)
    r = np.hypot(abs(a), abs(b))
    c = abs(a) / r
    s = (a / abs(a)) * np.conj(b) / r
    return c, s


def solve(A, precs, b: np.ndarray, tol: float = 1e-8, maxit: int = 200, scheme: str = "auto",
          eta: float = ETA, single_pass: bool = False, keep_basis: bool = False, gs_passes: int | None = None) -> Result:
    """A: sparse matrix (or anything with @); precs: list of callables r -> M_i^{-1} r."""
    t = len(precs)
    b = np.asarray(b, dtype=np.complex128)
    beta = np.linalg.norm(b)
    if beta == 0.0:
        return Result(np.zeros_like(b), 0, True, "ok", 0.0, 0.0)
    if scheme == "auto":
        scheme = "single" if t == 1 else ("cross" if t == 2 else "sum")
    passes = gs_passes if gs_passes is not None else (1 if single_pass else 2)

    V = [b / beta]
    Zs = []                 # accepted Z columns
    Hcols = []              # Hessenberg columns (length = nV at the time they were built + growth)
    cs, sn = [], []         # Givens rotations
    Rcols = []              # rotated columns (upper triangular part)
    g = [beta + 0.0j]
    history, ipcount = [], []
    src = [V[0]] * t
    converged = False
    status = "noconv"
    it = 0
    for it in range(1, maxit + 1):
        nip = 0
        Zk = [precs[i](src[i]) for i in range(t)]
        W = [A @ z for z in Zk]
        az = [np.linalg.norm(w) for w in W]        # deflation reference: ||A z_j||
        nold = len(V)
        Vm = np.array(V).T                           # dofs x nold
        Hold = np.zeros((nold, t), dtype=np.complex128)
        for _ in range(passes):
            for j in range(t):
                c = Vm.conj().T @ W[j]
                nip += nold
                W[j] = W[j] - Vm @ c
                Hold[:, j] += c
        new_v, new_from = [], []
        Rnew = np.zeros((t, t), dtype=np.complex128)
        accepted = []
        for j in range(t):
            w = W[j]
            for _ in range(passes):
                if new_v:
                    Vn = np.array(new_v).T               # accepted new vectors of this block
                    c = Vn.conj().T @ w
                    nip += len(new_v)
                    w = w - Vn @ c
                    Rnew[:len(new_v), j] += c
            rjj = np.linalg.norm(w)
            nip += 1
            if rjj == 0.0 or (new_v and rjj <= eta * az[j]):
                continue                             # deflated: Z_j dropped
            Rnew[len(new_v), j] = rjj
            new_v.append(w / rjj)
            new_from.append(j)
            accepted.append(j)
        ipcount.append(nip)
        if not accepted:
            status = "breakdown"
            it -= 1
            break
        # build the new Hessenberg columns (one per accepted Z column)
        for pos, j in enumerate(accepted):
            col = np.zeros(nold + len(accepted), dtype=np.complex128)
            col[:nold] = Hold[:, j]
            col[nold:nold + pos + 1] = Rnew[:pos + 1, j]
            Hcols.append(col)
            Zs.append(Zk[j])
            # rotate
            rc = col.copy()
            for i in range(len(cs)):
                a0, a1 = rc[i], rc[i + 1]
                rc[i] = cs[i] * a0 + sn[i] * a1
                rc[i + 1] = -np.conj(sn[i]) * a0 + cs[i] * a1
            cidx = len(cs)
            c_, s_ = _givens(rc[cidx], rc[cidx + 1])
            a0, a1 = rc[cidx], rc[cidx + 1]
            rc[cidx] = c_ * a0 + s_ * a1
            rc[cidx + 1] = 0.0
            cs.append(c_)
            sn.append(s_)
            g.append(0.0 + 0.0j)
            g0 = g[cidx]
            g[cidx] = c_ * g0
            g[cidx + 1] = -np.conj(s_) * g0
            Rcols.append(rc[:cidx + 1].copy())
        V.extend(new_v)
        rho = abs(g[-1])
        history.append(rho / beta)
        if rho / beta <= tol:
            converged = True
            status = "ok"
            break
        # next sources
        if scheme == "single":
            src = [new_v[0]] * t
        elif scheme == "cross":
            # preconditioner i takes the new vector made from Z column (i + 1) mod t
            # (for t = 2: the other preconditioner's), or the first survivor if deflated
            by_col = dict(zip(new_from, new_v))
            src = [by_col.get((i + 1) % t, new_v[0]) for i in range(t)]
        elif scheme == "sum":
            s = np.sum(new_v, axis=0)
            s = s / np.linalg.norm(s)
            src = [s] * t
        else:
            raise ValueError(scheme)

    nz = len(Zs)
    if nz == 0:
        x = np.zeros_like(b)
        return Result(x, 0, False, status, 1.0, 1.0, history, ipcount)
    Rm = np.zeros((nz, nz), dtype=np.complex128)
    for c, col in enumerate(Rcols):
        Rm[:c + 1, c] = col
    y = np.zeros(nz, dtype=np.complex128)
    gg = np.array(g[:nz])
    for i in range(nz - 1, -1, -1):
        y[i] = (gg[i] - Rm[i, i + 1:] @ y[i + 1:]) / Rm[i, i]
    Zm = np.array(Zs).T
    x = Zm @ y
    rel_exp = np.linalg.norm(b - A @ x) / beta
    res = Result(x, it, converged, status, abs(g[nz]) / beta, rel_exp, history, ipcount)
    if keep_basis:
        res.V = np.array(V).T
        res.Z = Zm
        nv = len(V)
        H = np.zeros((nv, nz), dtype=np.complex128)
        for c, col in enumerate(Hcols):
            H[:col.size, c] = col
        res.H = H
    return res
