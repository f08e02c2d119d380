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


def test_gpu_local_cpus_from_the_topology_table(monkeypatch):
    """The end-to-end host buffers are placed from the CPUs nvidia-smi lists as local to the GPU:
    the device is found by UUID, the CPU Affinity column parsed (ranges and lists) and intersected
    with the process's own CPUs; anything unexpected leaves the placement to the OS."""
    import os
    import types

    import torch

    table = ("\tGPU0\tGPU1\tNIC0\tCPU Affinity\tNUMA Affinity\tGPU NUMA ID\n"
             "GPU0\t X \tNV18\tSYS\t0-1,3\t0\t2\n"
             "GPU1\tNV18\t X \tSYS\t4-5\t1\t3\n"
             "NIC0\tSYS\tSYS\t X \t\t\t\n")

    def run(cmd, **kw):
        out = table if "topo" in cmd else "0, GPU-aaaa-0000\n1, GPU-bbbb-1111\n"
        return types.SimpleNamespace(stdout=out)

    monkeypatch.setattr(bench.subprocess, "run", run)
    monkeypatch.setattr(torch.cuda, "get_device_properties", lambda d: types.SimpleNamespace(uuid="bbbb-1111"))
    monkeypatch.setattr(os, "sched_getaffinity", lambda pid: {0, 1, 2, 3, 4})
    assert bench.gpu_local_cpus(0) == {4}  # GPU1's CPUs 4-5, of which this process may use 4
    monkeypatch.setattr(torch.cuda, "get_device_properties", lambda d: types.SimpleNamespace(uuid="aaaa-0000"))
    assert bench.gpu_local_cpus(0) == {0, 1, 3}
    monkeypatch.setattr(torch.cuda, "get_device_properties", lambda d: types.SimpleNamespace(uuid="cccc-2222"))
    assert bench.gpu_local_cpus(0) is None  # not listed
    monkeypatch.setattr(bench.subprocess, "run", lambda cmd, **kw: types.SimpleNamespace(stdout="no table here"))
    assert bench.gpu_local_cpus(0) is None


def test_workload_masses_follow_their_records():
    """A workload's mass is its lattice's recorded m0, or -Re(lambda_L) + the workload's own gap when
    it sets one (the 48^3 x 96 workload: edge + 1e-3)."""
    import json

    data = json.load(open(bench.WORKLOADS_JSON))
    for name, w in bench.WORKLOADS.items():
        m0, rec = bench.workload_m0(w)
        assert rec is data[w["m0_key"]] or rec == data[w["m0_key"]]
        if "gap" in w:
            assert abs(m0 - (-rec["lambda_L_m0_0"][0] + w["gap"])) < 1e-12
        else:
            assert m0 == float(rec["m0"])
    m48, rec48 = bench.workload_m0(bench.WORKLOADS["48x48x48x96"])
    assert abs(m48 - (-1.188968176108723 + 1e-3)) < 1e-9 and rec48["dims"] == [96, 48, 48, 48]


def test_spectral_edge_record_merges_into_the_workload_file(tmp_path, monkeypatch):
    """spectral_edge --record merges a record written by --out (on the GPU machine) into the workload
    file, leaving the other entries as they were."""
    import json
    import sys

    from paper_1303_1377_gb300 import spectral_edge

    wl = tmp_path / "workloads.json"
    wl.write_text(json.dumps({"a": {"m0": 1.0}, "b": {"m0": 2.0}}))
    rec = tmp_path / "edge.json"
    rec.write_text(json.dumps({"b": {"m0": -3.0, "lambda_L_m0_0": [3.0, 0.0]}}))
    monkeypatch.setattr(spectral_edge, "WORKLOADS", str(wl))
    monkeypatch.setattr(sys, "argv", ["spectral_edge", "--record", str(rec)])
    spectral_edge.main()
    out = json.loads(wl.read_text())
    assert out == {"a": {"m0": 1.0}, "b": {"m0": -3.0, "lambda_L_m0_0": [3.0, 0.0]}}
