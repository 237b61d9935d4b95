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
    else:
        assert value is None
    # every recorded capture: traffic at or below the algorithmic bytes (no re-reads)
    for kernel, per in t.items():
        for e in per.values():
            for mode in ("apply_p", "apply_s"):
                cap = sum(e["captured"][mode]) / len(e["captured"][mode])
                assert 0.5 * e["algorithmic"][mode] < cap <= 1.05 * e["algorithmic"][mode], (kernel, mode)
    assert bench.recorded_traffic("ildu0_apply", "no_such_workload") is None
    assert bench.recorded_traffic("no_such_kernel", bench.WORKLOAD) is None


def test_cpu_legs_run_the_oracle_on_all_host_cores(capsys):
    """The CPU baseline and the reference arm time the oracle's OpenMP build on
    every host core (single-thread sample beside it), on the ILDU0-form apply."""
    import argparse

    import oracle
    try:
        s, w = bench.workload_system("laplace16_sub8x8x4")
        d = bench.oracle_decomposition(s, w["grid"], w["sub"])
        out = bench.oracle_apply_baseline(d, w["grid"], 10 ** 6, budget_s=0.05)
        assert out["cores"] == bench.oracle_threads() == (os.cpu_count() or 1)
        assert out["single_thread"]["cores"] == 1 and out["value"] > 0 and out["kind"] == "oracle"
        bench.run_reference(argparse.Namespace(workload="laplace16_sub8x8x4", steps=2, warmup=1))
        line = json.loads(capsys.readouterr().out.strip().splitlines()[-1])
        assert line["impl"] == "reference" and line["cpu_baseline"]["cores"] == bench.oracle_threads()
        assert line["e2e"]["h2d_bytes_per_step"] == 0 and line["value"] > 0
    finally:
        oracle.set_threads(1)


def test_autotune_size_classes_and_pruning():
    """The tuner's size classes cover the batch once, smallest first, in equal
    counts; candidates too large for shared memory are pruned by the host-side
    plan before any device work."""
    from paper_2508_04917_gb300.autotune import candidates, size_classes
    systems = [synth.system(*sd, 5000 + i) for i, sd in enumerate(synth.ragged_batch(10))]
    cl = size_classes(systems, 3)
    assert sorted(i for c in cl for i in c) == list(range(10)) and [len(c) for c in cl] == [3, 3, 4]
    sizes = [[systems[i].n for i in c] for c in cl]
    assert max(sizes[0]) <= min(sizes[1]) and max(sizes[1]) <= min(sizes[2])
    s = synth.system(40, 40, 40, 1)
    cand = candidates(s, subs=((8, 8, 8), (40, 40, 40)), threads=(0, 128), factor_prec="f64")
    # a 40^3 box (64,000 rows) does not fit one block's shared memory
    assert cand == [((8, 8, 8), 0), ((8, 8, 8), 128)]


def test_autotune_pick_prefers_the_first_near_tie():
    from paper_2508_04917_gb300.autotune import pick
    trials = [dict(seconds=1.04), dict(seconds=1.00), dict(seconds=1.2)]
    assert pick(trials, tie=0.05) is trials[0]
    assert pick(trials, tie=0.01) is trials[1]


def test_source_hash_ignores_comments_only():
    import bench
    a = 'int f(int x) { // one\n  return x + 1; /* two */ }\nconst char* s = "a // b /* c */";\n'
    b = '/* header */\nint f(int x) {\n  return x + 1;   // other words\n}\nconst char* s = "a // b /* c */";'
    c = 'int f(int x) { return x + 2; }\nconst char* s = "a // b /* c */";'
    assert bench.strip_comments(a) == bench.strip_comments(b)
    assert bench.strip_comments(a) != bench.strip_comments(c)
    assert '"a // b /* c */"' in bench.strip_comments(a)
