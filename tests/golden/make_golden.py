"""Writes the stored expected values of the large workloads by running the CPU oracle.

Only oracle/ and the seeded input generators are used.  For each workload and right-hand
side it records the oracle's MPGMRES iteration count, residual history and explicit
residual at the workload's tolerance, and the solution at 512 seeded sample nodes (plus
its 2-norm) both at that tolerance and at a tight tolerance of 1e-10, the reference for
solution-error statements.

The tight solution is the oracle's MPGMRES at tol 1e-10, restarted on its residual (x += the
solve of A d = b - A x) until the explicit relative residual is at most 1e-10 (at most three
restarts); its explicit residual is stored with it.

usage: python tests/golden/make_golden.py k100_n256 [k400_n1024 ...] [--rhs 0,1,2] [--out f.json]
       python tests/golden/make_golden.py --merge k200_n512_b64 part0.json part1.json ...
"""
from __future__ import annotations

import argparse
import json
import os
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import hh_inputs  # noqa: E402
from oracle import solver  # noqa: E402

HERE = os.path.dirname(os.path.abspath(__file__))
NSAMPLE = 512


def sample_nodes(n: int) -> np.ndarray:
    rng = np.random.default_rng(123)
    m = n + 1
    idx = rng.choice(m * m, size=NSAMPLE - 4, replace=False)
    corners = np.array([0, n, n * m, m * m - 1])
    return np.sort(np.concatenate([idx, corners]))


def run(name: str, rhs_list=None, tight: float = 1e-10) -> dict:
    w = hh_inputs.workload(name)
    t0 = time.time()
    P = solver.Problem(w.k, w.n, w.strips, w.dirs)
    t_setup = time.time() - t0
    idx = sample_nodes(w.n)
    from oracle import mpgmres
    out = {"workload": name, "k": w.k, "n": w.n, "strips": w.strips, "dirs": w.dirs, "tol": w.tol,
           "tight_tol": tight, "sample_nodes": idx.tolist(), "oracle_setup_s": t_setup, "gs_passes": 2,
           "deflate_eta": mpgmres.ETA, "rhs": {}}
    rhs_list = range(w.nrhs) if rhs_list is None else rhs_list
    for r in rhs_list:
        b = P.rhs(w.sources[r])
        t1 = time.time()
        res = P.solve(b, tol=w.tol)
        t_solve = time.time() - t1
        res_t = P.solve(b, tol=tight)
        xt, restarts = res_t.x, 0
        rel_t = res_t.rel_res_explicit
        while rel_t > tight and restarts < 3:
            d = P.solve(b - P.A @ xt, tol=tight)
            xt = xt + d.x
            rel_t = float(np.linalg.norm(b - P.A @ xt) / np.linalg.norm(b))
            restarts += 1
        out["rhs"][str(r)] = {
            "iterations": res.iterations, "history": res.history, "rel_res_explicit": res.rel_res_explicit,
            "status": res.status, "solve_s": t_solve,
            "x_norm": float(np.linalg.norm(res.x)), "x_sample_re": res.x[idx].real.tolist(),
            "x_sample_im": res.x[idx].imag.tolist(),
            "tight_iterations": res_t.iterations, "tight_restarts": restarts, "tight_rel_res_explicit": rel_t,
            "tight_x_norm": float(np.linalg.norm(xt)), "tight_x_sample_re": xt[idx].real.tolist(),
            "tight_x_sample_im": xt[idx].imag.tolist(),
            "b_norm": float(np.linalg.norm(b)),
        }
        print(f"{name} rhs {r}: {res.iterations} it ({t_solve:.1f}s), tight {res_t.iterations} it", flush=True)
    return out


def merge(name: str, parts) -> None:
    """Joins files written with --rhs subsets of one workload into tests/golden/<name>.json."""
    data = None
    for p in parts:
        with open(p) as f:
            d = json.load(f)
        if data is None:
            data = d
        else:
            data["rhs"].update(d["rhs"])
    data["rhs"] = {k: data["rhs"][k] for k in sorted(data["rhs"], key=int)}
    path = os.path.join(HERE, f"{name}.json")
    with open(path, "w") as f:
        json.dump(data, f)
    print("wrote", path, "with", len(data["rhs"]), "right-hand sides")


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("names", nargs="+")
    ap.add_argument("--rhs", default=None)
    ap.add_argument("--out", default=None)
    ap.add_argument("--merge", action="store_true")
    a = ap.parse_args()
    if a.merge:
        merge(a.names[0], a.names[1:])
        return
    rl = None if a.rhs is None else [int(v) for v in a.rhs.split(",")]
    for name in a.names:
        data = run(name, rl)
        path = a.out or os.path.join(HERE, f"{name}.json")
        with open(path, "w") as f:
            json.dump(data, f)
        print("wrote", path)


if __name__ == "__main__":
    main()
