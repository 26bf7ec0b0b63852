"""bench.py's roofline traffic lookup (CPU): the committed ncu capture is used only for the tile
shape and K-slice reduction the autotuner chose, and only while the kernel sources it was
taken on are unchanged."""
import json
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


def test_traffic_matches_tuned_variant():
    d = json.load(open(os.path.join(ROOT, "profiles", "tc_line_gemm_traffic.json")))
    current = d["source_hash"] == bench.kernel_source_hash()
    for cap in d["captures"]:
        got = bench.ncu_traffic(cap["workload"], "tc", cap["complex_columns_per_cta"], cap["cluster"])
        # a capture taken on other kernel sources is not reported
        assert got == (float(cap["dram_bytes_per_step"]) if current else None)
        # the per-kernel figures add up to the step's figure
        assert abs(sum(cap["kernels"].values()) - cap["dram_bytes_per_step"]) < 1.0
        # at least the factor block (hi + lo, 16.8 MB at k=400) is read per step
        assert cap["dram_bytes_per_step"] > 16.8e6
    # a shape without a capture has no traffic figure
    assert bench.ncu_traffic(bench.WORKLOAD, "tc", 128, False) is None


def test_traffic_null_when_kernel_source_changed(monkeypatch):
    monkeypatch.setattr(bench, "kernel_source_hash", lambda extra=(): "0000000000000000")
    assert bench.ncu_traffic(bench.WORKLOAD, "tc", 64, False) is None
    assert bench.ncu_traffic(bench.WORKLOAD, "group") is None


def test_grouped_traffic_summary():
    """The grouped kernel's capture: the phases add up to the sweep, every twisted step reads at
    least its two factor blocks (2 x 16.8 MB of hi + lo at k=400), the one-shot corrections at
    least their 31-32 blocks, and the figure is reported only on the kernel sources it was taken on."""
    d = json.load(open(os.path.join(ROOT, "profiles", "tc_group_traffic.json")))
    w = d["workloads"]["k400_n1024"]
    ph = w["phases"]
    assert sum(v["launches"] for v in ph.values()) == w["launches_per_sweep"]
    assert abs(sum(v["dram_mb"] for v in ph.values()) * 1e6 - w["dram_bytes_per_sweep"]) < 1e6
    assert abs(w["dram_bytes_per_launch"] * w["launches_per_sweep"] - w["dram_bytes_per_sweep"]) < 1.0
    blk = 16.8e6
    for name in ("F1 forward", "F1 back"):
        v = ph[name]
        assert v["dram_mb"] * 1e6 / v["launches"] > 2 * blk * 0.95
    for name in ("F3 one-shot", "B2 one-shot"):
        assert ph[name]["dram_mb"] * 1e6 > 31 * blk * 0.95
    current = d["source_hash"] == bench.kernel_source_hash(("group.cu",))
    got = bench.ncu_traffic(bench.WORKLOAD, "group")
    assert got == (float(w["dram_bytes_per_launch"]) if current else None)
