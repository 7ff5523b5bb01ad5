"""Host logic of bench.py that needs no GPU: the clock record's parsing,
the traffic lookup's source check and the whole-job throughput."""
import json
import os

import bench


def _sampler_with(tmp_path, lines):
    s = bench.ClockSampler(0)
    s.path = str(tmp_path / "clocks.csv")
    with open(s.path, "w") as f:
        f.write("\n".join(lines) + "\n")
    s.proc = object()  # a sampler that ran
    return s


def test_clock_summary_median_and_reasons(tmp_path):
    s = _sampler_with(tmp_path, [
        "0, 2070, 2070, 900.1, 0x0, Not Active, Not Active, Not Active, Not Active",
        "0, 1980, 2070, 1390.0, 0x4, Not Active, Not Active, Not Active, Active",
        "0, 2070, 2070, 1200.0, 0x0, Not Active, Not Active, Not Active, Not Active",
        "garbage line",
        "0, [N/A], 2070, 1.0, 0x0, Not Active, Not Active, Not Active, Not Active",
    ])
    out = s.summary()
    assert out == {"sm_mhz": 2070.0, "sm_max_mhz": 2070.0, "samples": 3, "reasons": ["sw_power_cap"]}


def test_clock_summary_reports_slowdowns(tmp_path):
    s = _sampler_with(tmp_path, [
        "0, 1500, 2070, 800.0, 0x8, Active, Not Active, Not Active, Not Active",
        "0, 1400, 2070, 800.0, 0x8, Not Active, Active, Active, Not Active",
    ])
    out = s.summary()
    assert out["reasons"] == ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown"]
    assert out["sm_mhz"] == 1450.0


def test_clock_summary_without_a_sampler():
    assert bench.ClockSampler(0).summary() is None


def test_committed_traffic_follows_the_sources():
    p = os.path.join(bench.ROOT, "profiles", "traffic.json")
    with open(p) as f:
        d = json.load(f)
    name, k = next(iter(d["kernels"].items()))
    got = bench.committed_traffic(name, k["workload"])
    if d["source_hash"] == bench.kernel_source_hash():
        assert got == k["dram_bytes_per_launch"]
    else:
        assert got is None
    assert bench.committed_traffic(name, "another workload") is None
    assert bench.committed_traffic("no_such_kernel", k["workload"]) is None


def test_weak_value_counts_every_rank():
    # 2 ranks x 32 slices x 5 steps over the slowest rank's 4 s
    assert bench.weak_value(2, 32, 5, 4000.0) == 80.0
