"""Host logic of bench.py that needs no GPU: the clock summary that decides
whether a measurement is kept, the gating of the committed ncu traffic
record (same kernel sources and same workload only) and the peak loader's
fallback."""

import json
import os

import bench


def test_clock_summary_median_max_and_reasons():
    s = bench.ClockSampler(0)
    s.lines = [
        "2070, 2070, 900.1, 0x0, Not Active, Not Active, Not Active, Not Active",
        "2055, 2070, 1100.0, 0x4, Not Active, Not Active, Not Active, Active",
        "2070, 2070, 1200.0, 0x0, Not Active, Not Active, Not Active, Not Active",
        "garbage line",
        "[N/A], 2070, 1.0, 0x0, Not Active, Not Active, Not Active, Not Active",
    ]
    out = s.summary()
    assert out == {"sm_mhz": 2070.0, "sm_max_mhz": 2070.0, "reasons": ["sw_power_cap"], "samples": 3}
    s.lines = ["1500, 2070, 1.0, 0x8, Active, Not Active, Active, Not Active"]
    assert s.summary()["reasons"] == ["hw_slowdown", "sw_thermal_slowdown"]
    s.lines = []
    assert s.summary()["samples"] == 0


def test_traffic_only_for_its_sources_and_workload(monkeypatch):
    with open(os.path.join(bench.ROOT, "profiles", "ncu_traffic.json")) as fh:
        rec = json.load(fh)
    monkeypatch.setattr(bench, "source_digest", lambda: rec["source_digest"])
    monkeypatch.setattr(bench, "WORKLOAD", bench.WORKLOADS[rec["workload"]])
    for kernel, k in rec["kernels"].items():
        assert bench.ncu_traffic(kernel) == float(k["dram_bytes_per_launch"])
        assert k["dram_bytes_per_launch"] == k["dram_read"] + k["dram_write"]
    assert bench.ncu_traffic("no_such_kernel") is None
    other = next(w for w in bench.WORKLOADS if w != rec["workload"])
    monkeypatch.setattr(bench, "WORKLOAD", bench.WORKLOADS[other])
    assert bench.ncu_traffic("edge_qp") is None  # captured on another workload
    monkeypatch.setattr(bench, "WORKLOAD", bench.WORKLOADS[rec["workload"]])
    monkeypatch.setattr(bench, "source_digest", lambda: "0" * 16)
    assert bench.ncu_traffic("edge_qp") is None  # the kernels changed since the capture


def test_peaks_fall_back_without_the_measured_file(monkeypatch, tmp_path):
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    assert bench.load_peaks() == (6800.0, "fallback")
    (tmp_path / "MEASURED_PEAKS.json").write_text(json.dumps({"hbm_gbs": 6792.4}))
    assert bench.load_peaks() == (6792.4, "measured")
