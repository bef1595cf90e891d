"""Host-side pieces of bench.py (CPU only): the clock record's parsing of the
nvidia-smi samples, the code hash that keeps a recorded capture valid, and
the reference arm (the oracle on the host cores)."""
import json
import os

import bench


def _sampler(lines):
    s = bench.ClockSampler(0)
    s.lines = lines
    return s.summary()


def test_clock_summary_median_and_reasons():
    lines = ["0, 2070, 2070, 950.1, 0x0000000000000000, Not Active, Not Active, Not Active, Not Active",
             "0, 2060, 2070, 1200.0, 0x0000000000000004, Not Active, Not Active, Not Active, Active",
             "0, 2070, 2070, 1210.5, 0x0000000000000000, Not Active, Not Active, Not Active, Not Active"]
    s = _sampler(lines)
    assert s["sm_mhz"] == 2070.0 and s["sm_max_mhz"] == 2070.0
    assert s["reasons"] == ["sw_power_cap"] and s["samples"] == 3


def test_clock_summary_flags_thermal_slowdown_and_ignores_junk():
    lines = ["0, 1500, 2070, 1400.0, 0x40, Active, Not Active, Active, Not Active",
             "garbage", "0, [N/A], 2070, 0, 0x0, Not Active, Not Active, Not Active, Not Active"]
    s = _sampler(lines)
    assert s["reasons"] == ["hw_slowdown", "sw_thermal_slowdown"] and s["samples"] == 1


def test_clock_summary_without_samples():
    assert _sampler([])["reasons"] == ["unsampled"]


def test_clock_record_prefers_nvml_samples_of_the_timed_region():
    """NVML samples taken while the timed launches run make the record (their
    median and every throttle reason seen); without them the nvidia-smi
    samples over warm-up and timed region do."""
    smi = bench.ClockSampler(0)
    smi.lines = ["0, 1980, 2070, 900.0, 0x0, Not Active, Not Active, Not Active, Not Active"]
    nv = bench.NvmlClocks.__new__(bench.NvmlClocks)
    nv.samples, nv.max_mhz = [(2070.0, 0x0), (2055.0, 0x4), (2070.0, 0x0)], 2070.0
    r = bench.clocks_record(nv, smi)
    assert r["sm_mhz"] == 2070.0 and r["reasons"] == ["sw_power_cap"] and r["samples"] == 3
    assert r["source"].startswith("NVML")
    nv.samples = [(1500.0, 0x40 | 0x8)]
    assert bench.clocks_record(nv, smi)["reasons"] == ["hw_slowdown", "hw_thermal_slowdown"]
    nv.samples = []
    r = bench.clocks_record(nv, smi)
    assert r["sm_mhz"] == 1980.0 and r["source"].startswith("nvidia-smi")
    assert bench.clocks_record(None, smi)["sm_max_mhz"] == 2070.0


def test_nvml_index_follows_visible_devices(monkeypatch):
    monkeypatch.setenv("CUDA_VISIBLE_DEVICES", "3,5")
    assert bench.nvml_index(0) == 3 and bench.nvml_index(1) == 5
    monkeypatch.delenv("CUDA_VISIBLE_DEVICES")
    assert bench.nvml_index(2) == 2


def test_traffic_record_is_consistent_and_hash_ignores_comments(tmp_path, monkeypatch):
    """The traffic record names the code hash of its capture (the bench
    reports the DRAM traffic only while the sources still hash to it), and the
    hash does not move when only comments change."""
    pj = json.load(open(os.path.join(bench.ROOT, "profiles", "step_kernel_miscible128_traffic.json")))
    assert pj["dram_bytes_per_launch"] == pj["dram_bytes_read_per_launch"] + pj["dram_bytes_write_per_launch"]
    assert len(pj["source_hash"]) == 16 and int(pj["source_hash"], 16) >= 0
    csrc = os.path.join(bench.ROOT, "paper_0912_4230_gb300", "csrc")
    fake = tmp_path / "paper_0912_4230_gb300" / "csrc"
    fake.mkdir(parents=True)
    for f in ("lb_common.cuh", "lb_kernels.cuh", "lb_inst.cuh"):
        (fake / f).write_text(open(os.path.join(csrc, f)).read() + "\n// a comment\n/* another */\n")
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    commented = bench.kernel_source_hash()
    (fake / "lb_inst.cuh").write_text((fake / "lb_inst.cuh").read_text() + "int changed;\n")
    changed = bench.kernel_source_hash()
    monkeypatch.undo()
    assert commented == bench.kernel_source_hash() and changed != commented


def test_reference_arm_prints_one_line_on_rank_zero_only():
    """The oracle as the reference arm: one JSON line with the bench line's
    metric, unit and direction, its own cpu_baseline and e2e; other ranks
    print nothing and exit 0."""
    import subprocess
    import sys
    cmd = [sys.executable, os.path.join(bench.ROOT, "bench.py"), "--impl", "reference",
           "--steps", "1", "--warmup", "3"]
    out = subprocess.run(cmd, capture_output=True, text=True, timeout=600, check=True).stdout
    lines = [ln for ln in out.splitlines() if ln.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["metric"] == bench.METRIC and d["unit"] == "MLUPS"
    assert d["higher_is_better"] is True and d["value"] > 0 and d["steps"] == 1
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["value"] == d["value"]
    assert d["e2e"] == {"value": d["value"], "unit": "MLUPS", "h2d_bytes_per_step": 0,
                        "d2h_bytes_per_step": 0}
    # the same config as the default line of the CUDA arm
    assert d["config"] == bench.workload_config(1, bench.WORKLOAD, 128 ** 3, (128, 128, 128),
                                                bench.ALGO_BYTES_PER_LUP)
    assert "FP64" in d["arm"] and d["dtype"] == "f64"
    env = dict(os.environ, RANK="1", WORLD_SIZE="2")
    r = subprocess.run(cmd, capture_output=True, text=True, timeout=600, env=env)
    assert r.returncode == 0 and not [ln for ln in r.stdout.splitlines() if ln.startswith("{")]
