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
