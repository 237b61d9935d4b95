"""CPU checks of bench.py's pieces that need no GPU: the default workload is
the 160^3 layered system with 16x16x8 subdomains, and the committed
DRAM-traffic summary is used only while the kernel sources it was captured
from are unchanged."""
import json
import os

import bench
import synth

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_default_workload():
    assert bench.WORKLOAD in synth.WORKLOADS
    w = synth.WORKLOADS[bench.WORKLOAD]
    assert tuple(w["grid"]) == (160, 160, 160) and tuple(w["sub"]) == (16, 16, 8)


def test_traffic_summary_is_keyed_to_the_sources():
    t = json.load(open(os.path.join(ROOT, "profiles", "traffic.json")))
    entry = t["ildu0_apply"][bench.WORKLOAD]
    value = bench.recorded_traffic("ildu0_apply", bench.WORKLOAD)
    if entry["source_hash"] == bench.kernel_source_hash():
        assert value == float(entry["dram_bytes_per_launch"])
        # traffic at or below the algorithmic bytes: no re-reads
        alg = sum(entry["algorithmic_96"].values()) / 2
        cap = sum(entry["captured_96"].values()) / 2
        assert 0.5 * alg < cap <= 1.05 * alg
    else:
        assert value is None
    assert bench.recorded_traffic("ildu0_apply", "no_such_workload") is None
    assert bench.recorded_traffic("no_such_kernel", bench.WORKLOAD) is None
