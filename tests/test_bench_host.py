"""Host-side pieces of bench.py that need no GPU: the clock record and the shared metric name."""
import glob
import os
import tempfile

import bench


def test_clock_record_median_max_and_reasons():
    lines = [
        "0, 2070, 2070, 900.5, 0x0000000000000000, Not Active, Not Active, Not Active, Not Active",
        "0, 2055, 2070, 1390.0, 0x0000000000000004, Not Active, Not Active, Not Active, Active",
        "0, 2070, 2070, 1100.0, 0x0000000000000000, Not Active, Not Active, Not Active, Not Active",
        "garbage line",
        "0, [N/A], 2070, 0, 0x0, Not Active, Not Active, Not Active, Not Active",
    ]
    c = bench.ClockSampler.parse(lines)
    assert c == {"sm_mhz": 2070.0, "sm_max_mhz": 2070.0, "reasons": ["sw_power_cap"], "samples": 3}
    hot = bench.ClockSampler.parse(["0, 1500, 2070, 1400, 0x8, Not Active, Active, Not Active, Not Active"])
    assert hot["reasons"] == ["hw_thermal_slowdown"] and hot["sm_mhz"] == 1500.0


def test_clock_sampler_without_nvidia_smi_leaves_no_file(monkeypatch):
    monkeypatch.setenv("PATH", "/nonexistent")
    before = set(glob.glob(os.path.join(tempfile.gettempdir(), "clocks_gpu0_*.csv")))
    c = bench.ClockSampler(0)
    c.start()
    assert c.stop()["reasons"] == ["nvidia-smi unavailable"]
    assert set(glob.glob(os.path.join(tempfile.gettempdir(), "clocks_gpu0_*.csv"))) == before


def test_both_arms_share_metric_and_workload_text():
    w = bench.WORKLOADS["32x32x32x64"]
    assert bench.metric_name("32x32x32x64") == "solves/s to rel. residual 1e-10 (32^3x64, 12 point sources)"
    d = bench.workload_description("32x32x32x64", w, -0.931885)
    assert "32x32x32x64 lattice (L0=64)" in d and "12 point sources per step" in d and "N_v=20" in d
