"""Benchmark: time-to-1e-6 and solves/s of the multipreconditioned sweep solver at k=400.

Workload (default): k = 400, n = 1024 (1,050,625 unknowns), 32 strips of 32 node lines,
four double sweeps LR+RL+BT+TB as one sweep program per iteration, one Gaussian
source at (0.5, 0.5), tolerance 1e-6, complex64 strip factors and sweeps, complex128
Krylov side.  One step = one hh_solve from the assembled load vector to tol with the strip
factors already set up (the setup time is reported separately, like the FP64 form).

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]

Prints ONE JSON line (rank 0).  With N > 1 (torchrun) every rank solves its own copies
(replicas only: the method has no exchange step on one problem) and value is the total
number of solves of all ranks divided by the slowest rank's time.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import subprocess
import tempfile
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import hh_inputs  # noqa: E402

METRIC = "time-to-1e-6 residual & solves/s at k=400, FP32-sweep vs FP64; p50/p99 latency"
WORKLOAD = "k400_n1024"
L2_BYTES = 129 * 2 ** 20


def workload_desc(w) -> dict:
    return {
        "workload": f"{w.name}: k={w.k:g}, n={w.n} ({w.dofs:,} unknowns), {w.strips} strips of {w.n // w.strips} "
                    f"node lines, double sweeps {w.dirs} all in one sweep (every direction a column of one "
                    f"program of grouped steps, replayed as a CUDA graph), {w.nrhs} RHS (Gaussian sigma=0.05 at "
                    f"(0.5,0.5)), tol {w.tol:g}, complex64 factors+sweeps, complex128 Krylov",
        "k": w.k, "n": w.n, "strips": w.strips, "dirs": w.dirs, "nrhs": w.nrhs, "tol": w.tol,
        "l2": "inputs larger than L2: the complex64 factor store streamed by every sweep (33 blocks x 8.4 MB) "
              "and each 16.8 MB Krylov vector exceed the 129 MB L2; no flush between steps",
    }


# ---------------------------------------------------------------------- distributed helpers
def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def aggregate(elapsed_s: float, units: float, ws: int):
    """Max of the per-rank times and sum of the per-rank units (torch.distributed)."""
    if ws == 1:
        return elapsed_s, units
    import torch
    import torch.distributed as dist
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([elapsed_s], dtype=torch.float64, device=dev)
    u = torch.tensor([units], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    dist.all_reduce(u, op=dist.ReduceOp.SUM)
    return float(t.item()), float(u.item())


# ---------------------------------------------------------------------- clocks
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int = 0):
        self.index = index
        self.proc = None
        # raw samples: HH_CLOCKS_DIR if set, else the temporary directory (the JSON line carries
        # the summary)
        out_dir = os.environ.get("HH_CLOCKS_DIR", tempfile.gettempdir())
        self.path = os.path.join(out_dir, f"clocks_bench_{os.getpid()}.csv")

    def start(self):
        try:
            os.makedirs(os.path.dirname(self.path), exist_ok=True)
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"], stdout=self.fh,
                                         stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.fh.close()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            p = [v.strip() for v in line.split(",")]
            if len(p) < 9:
                continue
            try:
                sm.append(float(p[1]))
                smax.append(float(p[2]))
            except ValueError:
                continue
            for nm, v in zip(names, p[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": float(max(smax)), "reasons": sorted(reasons),
                "samples": len(sm)}


# ---------------------------------------------------------------------- peaks / traffic
def measured_peaks() -> dict:
    """HBM copy bandwidth and SM clock from MEASURED_PEAKS.json (else the fallback figures),
    plus the FP32 and FP64 ALU peaks derived from the unit counts at the maximum SM clock:
    152 SMs x 128 FP32 FMA lanes x 2 flops per clock, and the measured FP64 FMA rate."""
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        out = {"hbm_gbs": float(d["hbm_gbs"]), "sm_mhz": float(d.get("sm_max_mhz", 2070.0)), "src": "measured"}
    else:
        out = {"hbm_gbs": 6800.0, "sm_mhz": 2070.0, "src": "fallback"}
    out["fp32_alu_tflops"] = 152 * 128 * 2 * out["sm_mhz"] * 1e6 / 1e12
    # FP64: the nominal GB300 rate of the profiling recipe (FP64 FMA measured at 1.2 TFLOP/s)
    out["fp64_tflops"] = 1.25
    # TF32 dense tensor rate: the measured bf16 burst rate x the nominal TF32 / bf16 ratio
    bf16 = float(json.load(open(p))["bf16_tflops"]) if os.path.exists(p) else 1900.0
    out["tf32_tflops"] = bf16 * 1.1 / 2.25
    out["tf32_src"] = ("measured bf16 %.0f TFLOP/s (MEASURED_PEAKS.json) x nominal TF32/bf16 1.1/2.25" % bf16
                       if os.path.exists(p) else "fallback bf16 1900 TFLOP/s x 1.1/2.25")
    return out


# hh_opts.profile of the timed handles: every PROFILE_SAMPLE-th Arnoldi step (and sweep) runs
# eagerly with its kernel classes and GEMM launches timed by CUDA events, inside the timed
# region; the others replay their CUDA graphs
PROFILE_SAMPLE = 16


def kernel_source_hash(extra=()) -> str:
    h = hashlib.sha256()
    for f in ("gemm.cuh", "tc_gemm.cuh", "common.cuh") + tuple(extra):
        h.update(open(os.path.join(ROOT, "paper_2408_11929_gb300", "csrc", f), "rb").read())
    return h.hexdigest()[:16]


def ncu_traffic(workload: str, kind: str = "simt", bnc=None, cluster=None):
    """DRAM bytes of one wide sweep GEMM step (all its kernels), or the mean of one sweep's grouped
    launches (kind "group"), from the committed ncu summary, if it was taken on the current kernel
    source and, for the tensor-core step, on the tile shape and reduction the autotuner chose
    (else None)."""
    name = {"simt": "line_gemm_traffic.json", "tc": "tc_line_gemm_traffic.json", "group": "tc_group_traffic.json"}[kind]
    p = os.path.join(ROOT, "profiles", name)
    if not os.path.exists(p):
        return None
    d = json.load(open(p))
    if d.get("source_hash") != kernel_source_hash(("group.cu",) if kind == "group" else ()):
        return None
    if kind == "group":
        e = d.get("workloads", {}).get(workload)
        return None if e is None else float(e["dram_bytes_per_launch"])
    if kind == "tc":
        for cap in d.get("captures", []):
            if (cap["workload"] == workload and cap["complex_columns_per_cta"] == bnc
                    and bool(cap["cluster"]) == bool(cluster)):
                return float(cap["dram_bytes_per_step"])
        return None
    e = d.get("workloads", {}).get(workload)
    return None if e is None else float(e["dram_bytes_per_launch"])


def percentile(v, q):
    v = sorted(v)
    if not v:
        return None
    pos = (len(v) - 1) * q
    lo = int(pos)
    hi = min(lo + 1, len(v) - 1)
    return v[lo] + (v[hi] - v[lo]) * (pos - lo)


# ---------------------------------------------------------------------- oracle (CPU) baseline
CPU_SAMPLE_CODE = r"""
import json, sys, time, os
import numpy as np
sys.path.insert(0, %(root)r)
from oracle import fem, sweep
k, n, N, nsolve, steps, nv, t = %(k)r, %(n)r, %(N)r, %(nsolve)r, %(steps)r, %(nv)r, %(t)r
R = n // N
t0 = time.time()
D, glob = sweep.strip_matrix(k, n, 0, R - 1, "row", 1)
lu = sweep.BandLU(D, n + 2)
t_fact = time.time() - t0
A, K, M, MG = fem.global_system(k, n)
rng = np.random.default_rng(0)
r = rng.standard_normal(D.shape[0]) + 1j * rng.standard_normal(D.shape[0])
x = rng.standard_normal(A.shape[0]) + 1j * rng.standard_normal(A.shape[0])
dofs = A.shape[0]
V = np.linalg.qr(rng.standard_normal((dofs, nv)) + 1j * rng.standard_normal((dofs, nv)))[0]
W0 = rng.standard_normal((dofs, t)) + 1j * rng.standard_normal((dofs, t))
for step in range(steps):
    ts = time.time()
    t1 = time.time()
    for _ in range(nsolve):
        lu.solve(r)
    t_solve = (time.time() - t1) / nsolve
    t1 = time.time()
    for _ in range(3):
        A @ x
    t_mv = (time.time() - t1) / 3
    # one block Gram-Schmidt of t new columns against nv basis vectors, two passes (as the oracle)
    t1 = time.time()
    W = W0.copy()
    for _ in range(2):
        c = V.conj().T @ W
        W -= V @ c
    t_gs = time.time() - t1
    print(json.dumps(dict(step=step, t_fact=t_fact, t_solve=t_solve, t_mv=t_mv, t_gs=t_gs,
                          step_s=time.time() - ts)), flush=True)
"""


def oracle_sample(w, iters: int, nsolve: int = 6, threads: int = 1, steps: int = 1) -> list:
    """Times the oracle on a bounded sample of the workload in one subprocess with `threads`
    BLAS threads: one strip factorised (excluded, as the GPU step excludes setup), then per step
    nsolve strip solves (zgbtrs), 3 global matvecs and one block Gram-Schmidt of the t new
    columns against the basis size the solve averages over its iterations (two passes).  Each
    step's numbers scale to one full solve: iterations x (directions x (2N - 1) strip solves +
    directions matvecs + one block Gram-Schmidt)."""
    t_dirs = len(w.dirs.split("+"))
    nv = max(1, (1 + t_dirs * iters) // 2)  # average basis size over the iterations
    code = CPU_SAMPLE_CODE % dict(root=ROOT, k=w.k, n=w.n, N=w.strips, nsolve=nsolve, steps=steps, nv=nv, t=t_dirs)
    th = str(threads)
    env = dict(os.environ, OMP_NUM_THREADS=th, OPENBLAS_NUM_THREADS=th, MKL_NUM_THREADS=th)
    out = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, env=env, timeout=1800)
    if out.returncode != 0:
        raise RuntimeError(out.stderr[-2000:])
    res = []
    for line in out.stdout.strip().splitlines():
        if not line.startswith("{"):
            continue
        d = json.loads(line)
        per_iter = t_dirs * ((2 * w.strips - 1) * d["t_solve"] + d["t_mv"]) + d["t_gs"]
        d.update(iters=iters, nv=nv, per_iter_s=per_iter, solve_s_est=iters * per_iter)
        res.append(d)
    return res


# ---------------------------------------------------------------------- GPU arm
def golden(w):
    p = os.path.join(ROOT, "tests", "golden", f"{w.name}.json")
    return json.load(open(p)) if os.path.exists(p) else None


def run_gpu(args, ws, rank, local):
    import torch
    import __graft_entry__
    import paper_2408_11929_gb300 as hh

    __graft_entry__.build()
    torch.cuda.set_device(local)
    w = hh_inputs.workload(WORKLOAD)
    stream = torch.cuda.Stream()
    src = w.sources[0]
    peaks = measured_peaks()

    with torch.cuda.stream(stream):
        h = hh.Handle(w.k, w.n, w.strips, w.dirs, precision="fp32", profile=PROFILE_SAMPLE, stream=stream.cuda_stream,
                      bcr_depth=args.bcr_depth)
        setup_ms = h.stats()["setup_ms"]
        b = torch.from_numpy(h.assemble_rhs(src)).to(f"cuda:{local}")
        x = torch.zeros_like(b)
        for _ in range(args.warmup):
            _, res = h.solve(b, x, tol=w.tol)
        torch.cuda.synchronize()
        h.reset_stats()
        clk = ClockSampler(local)
        clk.start()
        if ws > 1:
            import torch.distributed as dist
            dist.barrier()
        torch.cuda.synchronize()
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps + 1)]
        ev[0].record(stream)
        iters = []
        for i in range(args.steps):
            _, res = h.solve(b, x, tol=w.tol)
            ev[i + 1].record(stream)
            iters.append(res.iterations)
        torch.cuda.synchronize()
        step_ms = [ev[i].elapsed_time(ev[i + 1]) for i in range(args.steps)]
        e0, e1 = ev[0], ev[-1]
        if ws > 1:
            dist.barrier()
        clocks = clk.stop()
        elapsed = e0.elapsed_time(e1) / 1000.0
        st = h.stats()
        status = res.status
        rel_exp = res.rel_res_explicit
        x_host = x.cpu().numpy()

        # end to end through the C ABI with host buffers (copies inside the timed region)
        b_host = b.cpu().numpy()
        xh = np.zeros_like(b_host)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(args.steps):
            h.solve(b_host, xh, tol=w.tol)
        e2e_s = time.perf_counter() - t0
        h.close()

    tmax, units = aggregate(elapsed, float(args.steps), ws)
    e2e_max, e2e_units = aggregate(e2e_s, float(args.steps), ws)
    out = None
    if rank == 0:
        nsw = max(1, st["sweep_launches"])
        sweep_ms = st["sweep_ms"] / nsw if st["sweep_ms"] > 0 else None
        ngm = max(1, st["gemm_launches"])
        gemm_ms = st["gemm_ms"] / ngm if st["gemm_ms"] > 0 else None
        gemm_flops = st["gemm_flops"] / ngm
        achieved = gemm_flops / (gemm_ms / 1e3) / 1e12 if gemm_ms else None
        step_total_ms = sum(step_ms)
        # Arnoldi steps per solve; with graphs on, the kernel classes are timed in every
        # PROFILE_SAMPLE-th step (eager) and scaled to all steps
        its = st["iterations_total"] / max(1, args.steps)
        avg = lambda ms, n: (ms / n) if n else 0.0
        phase = {"sweep": avg(st["sweep_ms"], st["sweep_launches"]) * its,
                 "spmv": avg(st["spmv_ms"], st["spmv_launches"]) * (its + 1),
                 "gram_schmidt": avg(st["gs_ms"], st["gs_launches"]) * its}
        # the two heaviest kernels: the wide sweep GEMM step (tensor cores) and the FP64
        # Gram-Schmidt inner products (two per step)
        gemm_total_ms = (gemm_ms or 0.0) * st["wide_steps"] * its * args.steps
        ngd = max(1, st["gsdot_launches"])
        gsdot_ms = st["gsdot_ms"] / ngd if st["gsdot_ms"] > 0 else None
        gsdot_flops = st["gsdot_flops"] / ngd
        gsdot_bytes = st["gsdot_bytes"] / ngd
        gsdot_gbs = gsdot_bytes / (gsdot_ms / 1e3) / 1e9 if gsdot_ms else None
        tc_on = bool(st["tensor_cores"])
        gemm_peak = peaks["tf32_tflops"] if tc_on else peaks["fp32_alu_tflops"]
        gemm_line = {
            "bound": "tensor" if tc_on else "alu",
            "kernel": ("tc_group_kernel (tcgen05 kind::tf32, 3 products per K step): the sweep's grouped "
                       "steps (two-task steps of the twisted strip solves, interface scans, one-shot corrections); "
                       "achieved = their algorithmic flops / their CUDA-event time, over every grouped launch of "
                       "the sampled sweeps" if st["twisted"] else
                       (("tc_line_gemm_kernel (tcgen05 kind::tf32, 3 products per K step)" +
                         (", K slices summed in a thread-block cluster" if st["tc_cluster"]
                          else " + split_reduce_kernel"))
                        if tc_on else "line_gemm_kernel<float> + split_reduce_kernel") + ": wide sweep GEMM step"),
            "achieved": achieved, "peak": gemm_peak, "unit": "TFLOP/s",
            "frac": (achieved / gemm_peak) if achieved else None,
            "traffic": (ncu_traffic(WORKLOAD, "group") if st["twisted"] else
                        ncu_traffic(WORKLOAD, "tc", st["tc_bnc"], st["tc_cluster"]) if tc_on
                        else ncu_traffic(WORKLOAD)),
            "algorithmic_flops_per_launch": gemm_flops, "avg_launch_ms": gemm_ms,
            "launches_timed": st["gemm_launches"],
            "share_of_step": gemm_total_ms / step_total_ms if step_total_ms > 0 else None,
            "autotuned": {"complex_columns_per_cta": st["tc_bnc"], "k_split": st["tc_nsplit"] or "fill SMs",
                          "k_slices_summed_in_cluster": bool(st["tc_cluster"]),
                          "us_when_tuned": st["tc_us"]} if tc_on else None,
            "peak_src": peaks["tf32_src"] if tc_on else
            "derived: 152 SMs x 128 FP32 FMA lanes x 2 flops x %.0f MHz" % peaks["sm_mhz"],
            "note": "algorithmic flops = 8 m^2 per complex column (complex multiply-adds); the tensor "
                    "cores execute three TF32 products per K step (hi*hi + hi*lo + lo*hi), so the "
                    "attainable fraction of the TF32 peak is at most 1/3"}
        gsdot_line = {
            "bound": "hbm",
            "kernel": "gst_dot_kernel<4>: Gram-Schmidt inner products on the tensor cores (exact integer "
                      "products of 7-bit slices in bf16, tcgen05 kind::f16, int64 sums; FP64-accurate)",
            "achieved": gsdot_gbs, "peak": peaks["hbm_gbs"], "unit": "GB/s",
            "frac": (gsdot_gbs / peaks["hbm_gbs"]) if gsdot_gbs else None, "traffic": None,
            "algorithmic_bytes_per_launch": gsdot_bytes, "avg_launch_ms": gsdot_ms,
            "launches_timed": st["gsdot_launches"],
            "share_of_step": (gsdot_ms or 0.0) * 2 * its * args.steps / step_total_ms if step_total_ms > 0 else None,
            "peak_src": "measured HBM copy bandwidth (MEASURED_PEAKS.json)",
            "note": "algorithmic bytes = 32 per node and basis vector (its eight digit planes in bf16) "
                    "+ 16 t per node (the new columns in FP64, sliced into digits inside the kernel; read "
                    "once per plane, twice in all), each read once; the FP64-pipe form "
                    "of the same products ran at 1.1-1.4 TFLOP/s, bound by GB300's FP64 rate"}
        ranked = sorted([gemm_line, gsdot_line], key=lambda r: -(r["share_of_step"] or 0))
        dominant, others = ranked[0], ranked[1:]
        g = golden(w)
        err = None
        iters_oracle = None
        oracle_cmp = None
        if g is not None:
            idx = np.array(g["sample_nodes"])
            r0 = g["rhs"]["0"]
            xt = np.array(r0["tight_x_sample_re"]) + 1j * np.array(r0["tight_x_sample_im"])
            xs = np.array(r0["x_sample_re"]) + 1j * np.array(r0["x_sample_im"])
            err = float(np.linalg.norm(x_host[idx] - xt) / np.linalg.norm(xt))
            iters_oracle = r0["iterations"]
            oracle_cmp = {
                "vs_oracle_same_tol": float(np.linalg.norm(x_host[idx] - xs) / np.linalg.norm(xs)),
                "vs_oracle_tight": err,
                "oracle_own_stop_error": float(np.linalg.norm(xs - xt) / np.linalg.norm(xt)),
                "oracle_rel_res_explicit": r0["rel_res_explicit"],
                "sample": "%d stored nodes (tests/golden)" % len(idx)}
        out = {
            "metric": METRIC, "value": units / tmax, "unit": "solves/s", "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": tmax / args.steps * 1e3, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "c64 sweeps + c128 Krylov", "data": "synthetic",
            "config": workload_desc(w),
            "time_to_tol_ms": tmax / args.steps * 1e3, "iterations": iters[-1], "iterations_oracle": iters_oracle,
            "status": hh.STATUS_NAMES[status], "rel_res_explicit": rel_exp, "setup_ms": setup_ms,
            "error_vs_oracle_tight": err,
            "error_vs_oracle": oracle_cmp,
            "setup": {"ms": setup_ms, "flops": st["setup_flops"],
                      "tflops": st["setup_flops"] / (setup_ms / 1e3) / 1e12 if setup_ms else None,
                      "frac_of_tf32_peak": (st["setup_flops"] / (setup_ms / 1e3) / 1e12 / peaks["tf32_tflops"])
                      if setup_ms else None,
                      "setup_plus_solve_ms": setup_ms + tmax / args.steps * 1e3,
                      "newton_schulz_blocks": st["ns_blocks"], "newton_schulz_iterations": st["ns_iterations"]},
            "roofline": dominant,
            "roofline_others": others,
            "phase_roofline": {
                "sweep": {"ms_per_launch": sweep_ms, "bytes_per_launch": st["sweep_bytes"] / nsw,
                          "gbs": (st["sweep_bytes"] / nsw) / (sweep_ms / 1e3) / 1e9 if sweep_ms else None,
                          "hbm_frac": ((st["sweep_bytes"] / nsw) / (sweep_ms / 1e3) / 1e9 / peaks["hbm_gbs"]) if sweep_ms else None},
                "spmv": {"gbs": st["spmv_bytes"] / (st["spmv_ms"] / 1e3) / 1e9 if st["spmv_ms"] > 0 else None,
                         "hbm_frac": (st["spmv_bytes"] / (st["spmv_ms"] / 1e3) / 1e9 / peaks["hbm_gbs"]) if st["spmv_ms"] > 0 else None},
                "gram_schmidt": {"gbs": st["gs_bytes"] / (st["gs_ms"] / 1e3) / 1e9 if st["gs_ms"] > 0 else None,
                                 "hbm_frac": (st["gs_bytes"] / (st["gs_ms"] / 1e3) / 1e9 / peaks["hbm_gbs"]) if st["gs_ms"] > 0 else None},
                "hbm_peak_gbs": peaks["hbm_gbs"]},
            "latency_ms": {"p50": percentile(step_ms, 0.5), "p99": percentile(step_ms, 0.99),
                           "samples": len(step_ms), "kind": "closed loop, one solve at a time"},
            "e2e": {"value": e2e_units / e2e_max, "unit": "solves/s", "h2d_bytes_per_step": int(b_host.nbytes),
                    "d2h_bytes_per_step": int(xh.nbytes)},
            "gpu_launches": int(st["kernel_launches"]),
            "clocks": clocks,
            "phase_ms_per_step": {**phase, "how": f"class time per timed launch (every {PROFILE_SAMPLE}th Arnoldi "
                                              "step runs eagerly with CUDA events) x launches per step"},
            "arnoldi_steps_per_step": its,
        }
    return out


def run_other_precision(w, local, precision: str, warmup: int, steps: int) -> dict:
    """The same solve with another precision of the strip factors and sweeps: "fp64" (complex128,
    the FP32-vs-FP64 part of the metric) or "bf16" (bf16 factors and products, the
    lower-precision subsolves of Section 5): setup time, then the mean of `steps` timed solves
    after `warmup` untimed ones (CUDA events on the handle's stream), the iteration count,
    the explicit residual and the error against the oracle's tight solution (stored nodes)."""
    import torch
    import paper_2408_11929_gb300 as hh
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        h = hh.Handle(w.k, w.n, w.strips, w.dirs, precision=precision, stream=stream.cuda_stream)
        setup_ms = h.stats()["setup_ms"]
        b = torch.from_numpy(h.assemble_rhs(w.sources[0])).to(f"cuda:{local}")
        x = torch.zeros_like(b)
        for _ in range(warmup):
            h.solve(b, x, tol=w.tol)
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(steps):
            _, res = h.solve(b, x, tol=w.tol)
        e1.record(stream)
        torch.cuda.synchronize()
        x_host = x.cpu().numpy()
        h.close()
    out = {"ms_per_solve": e0.elapsed_time(e1) / steps, "timed_solves": steps, "iterations": res.iterations,
           "setup_ms": setup_ms, "rel_res_explicit": res.rel_res_explicit}
    g = golden(w)
    if g is not None:
        idx = np.array(g["sample_nodes"])
        r0 = g["rhs"]["0"]
        xt = np.array(r0["tight_x_sample_re"]) + 1j * np.array(r0["tight_x_sample_im"])
        out["error_vs_oracle_tight"] = float(np.linalg.norm(x_host[idx] - xt) / np.linalg.norm(xt))
    return out


SERVE_MAXIT = 40  # iteration cap of a served request (the server reserves memory for it)


def run_serving(nreq: int, rate_hz, seed: int = 0) -> dict:
    """The mixed-k request stream: nreq requests (k uniform in [50, 400], n = ceil(2.5k/32)*32,
    strips of 32 node lines, one Gaussian each, tol 1e-6) arriving as a Poisson stream of
    rate_hz (None: all at once, which measures the capacity), through one hh_server (complex64
    sweeps on the tensor cores, 2 slots per problem, iteration cap SERVE_MAXIT).  Latency =
    submission to completion (queueing, setup of an uncached problem and the solve);
    throughput = requests / (last completion - first arrival).  The stream's problems are nearly
    all distinct (each solved about once), so the server keeps block Thomas (twisted = 0): the
    twisted strip solves' extra setup (58 ms at k = 400) exceeds what they save in one solve."""
    import paper_2408_11929_gb300 as hh
    reqs = hh_inputs.serving_stream(nreq, seed=seed, rate_hz=rate_hz if rate_hz else 1e12)
    xs = [np.zeros((q["n"] + 1) ** 2, dtype=np.complex128) for q in reqs]
    done, tickets = {}, []
    with hh.Server(precision="fp32", serve_slots=2, maxit=SERVE_MAXIT, twisted=0) as srv:
        t0 = time.perf_counter()
        i = 0
        while len(done) < len(reqs):
            now = time.perf_counter() - t0
            while i < len(reqs) and reqs[i]["t_arrive"] <= now:
                q = reqs[i]
                tickets.append(srv.submit(q["k"], q["n"], q["strips"], q["sources"], xs[i], tol=1e-6))
                i += 1
            for j, t in enumerate(tickets):
                if j not in done:
                    st, res = srv.poll(t)
                    if st != hh.HH_EPENDING:
                        done[j] = (st, res, time.perf_counter() - t0)
            time.sleep(0.0005)
        stats = srv.stats()
    lat = [done[j][1].t_solve_ms for j in range(len(reqs))]
    t_end = max(done[j][2] for j in range(len(reqs)))
    return {
        "nreq": nreq, "rate_hz": rate_hz if rate_hz else "all at t=0 (capacity)", "seed": seed,
        "p50_ms": percentile(lat, 0.5), "p99_ms": percentile(lat, 0.99), "mean_ms": float(np.mean(lat)),
        "solves_per_s": nreq / (t_end - reqs[0]["t_arrive"]),
        "all_ok": all(done[j][0] == hh.HH_OK for j in range(len(reqs))),
        "max_rel_res_explicit": max(done[j][1].rel_res_explicit for j in range(len(reqs))),
        "iterations_mean": float(np.mean([done[j][1].iterations for j in range(len(reqs))])),
        "setups": stats["setups"], "cache_hits": stats["cache_hits"], "evictions": stats["evictions"],
        "cache_hit_rate": stats["cache_hits"] / max(1, stats["cache_hits"] + stats["setups"]),
        "maxit": SERVE_MAXIT, "makespan_s": t_end - reqs[0]["t_arrive"],
        "setup_ms_total": stats["setup_ms"], "k_range": [50, 400], "n_range": [128, 1024],
        "kind": "open loop, Poisson arrivals, mixed k; latency includes queueing and the setup of uncached problems"}


def run_batch(name: str = "k200_n512_b64") -> dict:
    """The batching configuration: all right-hand sides of the workload in one hh_solve_batch
    (complex64 sweeps on the tensor cores; every sweep serves all columns and directions).
    One warm-up batch, then one timed batch with CUDA events."""
    import torch
    import paper_2408_11929_gb300 as hh
    w = hh_inputs.workload(name)
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        t0 = time.perf_counter()
        # every 8th step sampled: the batch's GEMM-step rate is taken while most slots are
        # still active (later steps have fewer columns)
        h = hh.Handle(w.k, w.n, w.strips, w.dirs, precision="fp32", profile=8, stream=stream.cuda_stream)
        setup_s = time.perf_counter() - t0
        B = torch.cat([torch.from_numpy(h.assemble_rhs(src)) for src in w.sources]).cuda()
        X = torch.zeros_like(B)
        h.solve_batch(B, w.nrhs, X, tol=w.tol)
        torch.cuda.synchronize()
        h.reset_stats()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        _, res = h.solve_batch(B, w.nrhs, X, tol=w.tol)
        e1.record(stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1)
        st = h.stats()
        h.close()
    its = [r.iterations for r in res]
    ng = max(1, st["gemm_launches"])
    gemm_ms = st["gemm_ms"] / ng if st["gemm_ms"] > 0 else None
    gemm_tf = (st["gemm_flops"] / ng) / (gemm_ms / 1e3) / 1e12 if gemm_ms else None
    peaks = measured_peaks()
    return {"workload": name, "k": w.k, "n": w.n, "strips": w.strips, "nrhs": w.nrhs, "tol": w.tol,
            "ms_per_batch": ms, "solves_per_s": w.nrhs / (ms / 1e3), "setup_s": setup_s,
            "iterations_mean": float(np.mean(its)), "iterations_max": int(max(its)),
            "all_ok": all(r.status == hh.HH_OK for r in res),
            "max_rel_res_explicit": max(r.rel_res_explicit for r in res),
            "gemm_step": {"avg_launch_ms": gemm_ms, "tflops_algorithmic": gemm_tf,
                          "frac_of_tf32_peak": gemm_tf / peaks["tf32_tflops"] if gemm_tf else None,
                          "launches_timed": st["gemm_launches"], "tile": st["tc_bnc"], "k_split": st["tc_nsplit"]}}


def run_candidates(args):
    """Whole 4-column BT double sweeps (k = 0.39 n) for every forced candidate of the
    tensor-core step's autotuner (hh_opts.autotune = -(1 + cand)): 3 warm-up sweeps, then the
    mean of 20, CUDA events on the handle's stream."""
    import torch
    import __graft_entry__
    import paper_2408_11929_gb300 as hh
    __graft_entry__.build()
    k = 400.0 * args.n / 1024
    dofs = (args.n + 1) ** 2
    r = torch.from_numpy(np.ascontiguousarray(hh_inputs.random_vector(dofs, 4, seed=1).ravel())).cuda()
    z = torch.zeros_like(r)
    out = {}
    for cand in range(21):
        stream = torch.cuda.Stream()
        with torch.cuda.stream(stream):
            with hh.Handle(k, args.n, args.strips, precision="fp32", autotune=-(1 + cand),
                           stream=stream.cuda_stream) as h:
                for _ in range(3):
                    h.apply_preconditioner("BT", r, 4, z)
                torch.cuda.synchronize()
                e0 = torch.cuda.Event(enable_timing=True)
                e1 = torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                for _ in range(20):
                    h.apply_preconditioner("BT", r, 4, z)
                e1.record(stream)
                torch.cuda.synchronize()
                out[cand] = e0.elapsed_time(e1) / 20
    print(json.dumps({"mode": "candidates", "n": args.n, "strips": args.strips, "ms_per_sweep": out}), flush=True)


def run_fd_table(args):
    """The paper's own setting (five-point finite differences, 8 overlapping strips, the paper's
    source, tol 1e-6) for Table 1's preconditioner combinations: iterations and GPU times, to set
    beside the paper's printed counts.  One line per (k, combination)."""
    import torch
    import __graft_entry__
    import paper_2408_11929_gb300 as hh
    __graft_entry__.build()
    n, N = args.n, 8
    for k in (50.0, 100.0):
        # Section 4's source 3e4 exp(-200 k |x - (1/2, 1/2)|^2): a Gaussian with sigma^2 = 1/(400 k)
        src = np.array([[0.5, 0.5, (1.0 / (400.0 * k)) ** 0.5, 3e4, 0.0]])
        for dirs, double in (("LR", True), ("LR+BT", True), ("LR+RL", False), ("LR+RL+BT+TB", False),
                             ("LR+RL+BT+TB", True)):
            with hh.Handle(k, n, N, dirs, discretization=hh.HH_DISC_FD, single_sweep=0 if double else 1,
                           maxit=300) as h:
                b = torch.from_numpy(h.assemble_rhs(src)).cuda()
                h.solve(b, tol=1e-6)  # warm-up: graph capture
                torch.cuda.synchronize()
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record()
                x, res = h.solve(b, tol=1e-6)
                e1.record()
                torch.cuda.synchronize()
                st = h.stats()
            print(json.dumps({"mode": "fd", "k": k, "n": n, "strips": N, "dirs": dirs,
                              "sweeps": "double" if double else "single", "iterations": res.iterations,
                              "status": hh.STATUS_NAMES[res.status], "rel_res_explicit": res.rel_res_explicit,
                              "setup_ms": st["setup_ms"], "solve_ms": e0.elapsed_time(e1)}), flush=True)


def run_sweep_only(args):
    """One direction's double sweep on 4 columns (the column count of one 4-direction solve
    iteration), k = 0.39 n, timed with CUDA events on the launching stream."""
    import torch
    import __graft_entry__
    import paper_2408_11929_gb300 as hh
    __graft_entry__.build()
    k = 400.0 * args.n / 1024
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        extra = {} if args.twisted is None else {"twisted": args.twisted}
        h = hh.Handle(k, args.n, args.strips, "LR+RL+BT+TB", precision=args.precision, profile=1,
                      autotune=args.autotune, bcr_depth=args.bcr_depth,
                      stream=stream.cuda_stream, **extra)
        dofs = (args.n + 1) ** 2
        r = torch.from_numpy(np.ascontiguousarray(hh_inputs.random_vector(dofs, 4, seed=1).ravel())).cuda()
        z = torch.zeros_like(r)
        for _ in range(args.warmup):
            h.apply_preconditioner("BT", r, 4, z)
        h.reset_stats()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(args.steps):
            h.apply_preconditioner("BT", r, 4, z)
        e1.record(stream)
        torch.cuda.synchronize()
        st = h.stats()
        h.close()
    ms = st["sweep_ms"] / max(1, st["sweep_launches"])
    print(json.dumps({"mode": "sweep", "n": args.n, "strips": args.strips, "precision": args.precision,
                      "bcr_depth": st["bcr_depth"], "twisted": st["twisted"], "setup_ms": st["setup_ms"],
                      "sweep_ms": ms, "steps_per_launch": st["sweep_steps"],
                      "us_per_step": ms * 1e3 / st["sweep_steps"],
                      "GBps": st["sweep_bytes"] / max(1, st["sweep_launches"]) / (ms / 1e3) / 1e9,
                      "total_ms": e0.elapsed_time(e1),
                      "gemm_launches_per_sweep": st["gemm_launches"] / max(1, st["sweep_launches"]),
                      "gemm_us_per_launch": st["gemm_ms"] * 1e3 / max(1, st["gemm_launches"]),
                      "gemm_tflops": (st["gemm_flops"] / (st["gemm_ms"] / 1e3) / 1e12) if st["gemm_ms"] > 0 else None,
                      "gemm_share_of_sweep": st["gemm_ms"] / st["sweep_ms"] if st["sweep_ms"] > 0 else None}),
          flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu", action="store_true", help="skip the oracle CPU baseline")
    ap.add_argument("--no-fp64", action="store_true", help="skip the FP64 comparison solve")
    ap.add_argument("--no-batch", action="store_true", help="skip the 64-right-hand-side batch")
    ap.add_argument("--serve-nreq", type=int, default=500, help="requests of the mixed-k serving stream (0: skip)")
    ap.add_argument("--serve-rate", type=float, default=0.0,
                    help="--mode serve: Poisson arrival rate (1/s); 0: all at once (capacity)")
    ap.add_argument("--mode", default="solve", choices=["solve", "sweep", "serve", "solve1", "candidates", "fd"],
                    help="sweep: time hh_apply_preconditioner alone (4 columns) -- the profiling case")
    ap.add_argument("--n", type=int, default=1024)
    ap.add_argument("--strips", type=int, default=32)
    ap.add_argument("--precision", default="fp32")
    ap.add_argument("--bcr-depth", type=int, default=-1,
                    help="cyclic-reduction depth of the strip solves (-1: autotuned, 0: block Thomas)")
    ap.add_argument("--twisted", type=int, default=None,
                    help="--mode sweep/solve1: hh_opts.twisted (1: twisted strip solves, -1: timed against "
                         "block Thomas, 0: off; default: the library's)")
    ap.add_argument("--autotune", type=int, default=0,
                    help="--mode solve1/sweep: hh_opts.autotune (0: the default tile; -(1 + 7 shape + variant): "
                         "one candidate, e.g. -13 = 32 columns, 4 K slices summed in a cluster)")
    args = ap.parse_args()
    if args.mode == "sweep":
        run_sweep_only(args)
        return
    if args.mode == "candidates":
        run_candidates(args)
        return
    if args.mode == "solve1":
        # setup and one solve of the default workload, nothing else: the profiling case
        import torch
        import __graft_entry__
        import paper_2408_11929_gb300 as hh
        __graft_entry__.build()
        w = hh_inputs.workload(WORKLOAD)
        # no autotuning: under a profiler the tuner's timings are blurred by the per-launch
        # overhead; --autotune forces the candidate the tuner picks in the live bench
        extra = {} if args.twisted is None else {"twisted": args.twisted}
        with hh.Handle(w.k, w.n, w.strips, w.dirs, precision="fp32", autotune=args.autotune, **extra) as h:
            b = torch.from_numpy(h.assemble_rhs(w.sources[0])).cuda()
            x, res = h.solve(b, tol=w.tol)
            torch.cuda.synchronize()
            st = h.stats()
        print(json.dumps({"mode": "solve1", "iterations": res.iterations, "status": hh.STATUS_NAMES[res.status],
                          "rel_res_explicit": res.rel_res_explicit, "kernel_launches": st["kernel_launches"],
                          "bcr_depth": st["bcr_depth"], "twisted": st["twisted"], "sweep_steps": st["sweep_steps"]}),
              flush=True)
        return
    if args.mode == "fd":
        run_fd_table(args)
        return
    if args.mode == "serve":
        import __graft_entry__
        __graft_entry__.build()
        print(json.dumps({"mode": "serve", **run_serving(args.serve_nreq, args.serve_rate)}), flush=True)
        return
    ws, rank, local = dist_env()
    w = hh_inputs.workload(WORKLOAD)

    if args.impl == "reference":
        if rank != 0:
            return
        g = golden(w)
        iters = g["rhs"]["0"]["iterations"] if g else 20
        t0 = time.time()
        samples = oracle_sample(w, iters, nsolve=2, steps=args.warmup + args.steps)[args.warmup:]
        est = [d["solve_s_est"] for d in samples]
        v = len(est) / sum(est)
        step_ms = float(np.mean([d["step_s"] for d in samples])) * 1e3
        sample = (f"per step: 2 strip solves (zgbtrs) of a factorised 32-line k=400 strip, 3 global matvecs and "
                  f"one two-pass block Gram-Schmidt of {len(w.dirs.split('+'))} columns against "
                  f"{samples[0]['nv']} basis vectors (the solve's average), scaled to a full solve = {iters} "
                  f"iterations x ({len(w.dirs.split('+'))} directions x {2 * w.strips - 1} strip solves + matvecs "
                  f"+ Gram-Schmidt); the strip factorisation ({samples[0]['t_fact']:.1f} s, once) is excluded like "
                  f"the GPU setup; single thread")
        line = {"metric": METRIC, "value": v, "unit": "solves/s", "n_gpus": ws, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": step_ms, "higher_is_better": True, "scaling": "weak",
                "vs_baseline": None, "dtype": "c128", "data": "synthetic", "config": workload_desc(w),
                "impl": "reference",
                "solve_s_estimated_per_step": float(np.mean(est)),
                "note": "ms_per_step is the wall time of one sample step; value = solves/s scaled from the samples",
                "cpu_baseline": {"value": v, "unit": "solves/s", "cores": 1, "kind": "oracle", "sample": sample},
                "e2e": {"value": v, "unit": "solves/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
                "wall_s": time.time() - t0}
        print(json.dumps(line), flush=True)
        return

    if ws > 1:
        import torch
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    out = run_gpu(args, ws, rank, local)
    if rank == 0:
        if not args.no_batch:
            out["batch"] = run_batch()
        if args.serve_nreq > 0:
            # capacity (every request at t = 0), then Poisson streams at 0.7 and 0.9 of it
            cap = run_serving(args.serve_nreq, None)
            runs = {"capacity": cap}
            for f in (0.7, 0.9):
                runs[f"poisson_{f:.1f}x_capacity"] = run_serving(args.serve_nreq, f * cap["solves_per_s"])
            out["serving"] = runs
            out["latency_ms"]["serving_p50"] = runs["poisson_0.7x_capacity"]["p50_ms"]
            out["latency_ms"]["serving_p99"] = runs["poisson_0.7x_capacity"]["p99_ms"]
        if not args.no_fp64:
            out["fp64"] = run_other_precision(w, local, "fp64", warmup=1, steps=2)
            out["fp32_speedup_vs_fp64"] = out["fp64"]["ms_per_solve"] / out["ms_per_step"]
        out["bf16"] = run_other_precision(w, local, "bf16", warmup=2, steps=5)
        if not args.no_cpu:
            its = out["iterations_oracle"] or out["iterations"]
            d = oracle_sample(w, its, nsolve=6, steps=1)[0]
            out["cpu_baseline"] = {
                "value": 1.0 / d["solve_s_est"], "unit": "solves/s", "cores": 1, "kind": "oracle",
                "sample": (f"one 32-line k=400 strip factorised (zgbtrf, {d['t_fact']:.1f} s, excluded like the GPU "
                           f"setup), 6 timed strip solves ({d['t_solve'] * 1e3:.0f} ms each), 3 global matvecs "
                           f"({d['t_mv'] * 1e3:.0f} ms) and one two-pass block Gram-Schmidt of 4 columns against "
                           f"{d['nv']} vectors ({d['t_gs'] * 1e3:.0f} ms), scaled to {d['iters']} iterations x "
                           f"(4 directions x {2 * w.strips - 1} strip solves + matvecs + Gram-Schmidt); single thread "
                           f"(OMP/OPENBLAS_NUM_THREADS=1)"),
                "host_cores_available": os.cpu_count()}
            dn = oracle_sample(w, its, nsolve=4, threads=os.cpu_count() or 1, steps=1)[0]
            out["cpu_baseline_all_cores"] = {"value": 1.0 / dn["solve_s_est"], "unit": "solves/s",
                                             "cores": os.cpu_count(), "kind": "oracle",
                                             "sample": "as cpu_baseline with BLAS/LAPACK threads = all host cores"}
        print(json.dumps(out), flush=True)
    if ws > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
