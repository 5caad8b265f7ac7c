"""Host logic of bench.py, on the CPU: the run contract's defaults, the
clock summary taken from nvidia-smi samples, and the rule that reports the
smoother's DRAM traffic only while the profiled kernel source is unchanged."""
import os
import shutil

import pytest

import bench

MARK = "// ---------------------------------------------------------------- transfers"


def test_defaults_are_one_gpu_and_enough_warmup():
    a = bench.parse_args([])
    assert a.gpus == 1 and a.warmup >= 3 and a.steps >= 1 and a.impl == "ours"
    assert not a.no_cpu_baseline and not a.no_request_loop


def _row(sm, mx, reasons=()):
    names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
    flags = ["Active" if n in reasons else "Not Active" for n in names]
    return ["0", str(sm), str(mx), "812.40", "0x0000000000000000"] + flags


def test_clock_summary():
    rows = [_row(2070, 2070), _row(1980, 2070, ("sw_power_cap",)), _row(2070, 2070),
            ["0", "[N/A]", "2070", "[N/A]", "0x0", "Not Active", "Not Active", "Not Active", "Not Active"],
            ["garbage"]]
    c = bench.ClockSampler.summarize(rows)
    assert c["samples"] == 4  # the short row is dropped
    assert c["sm_mhz"] == 2070.0  # median of the three numeric samples
    assert c["sm_max_mhz"] == 2070.0
    assert c["reasons"] == ["sw_power_cap"]  # "Not Active" is not active
    assert bench.ClockSampler.summarize([]) is None
    hot = bench.ClockSampler.summarize([_row(1500, 2070, ("hw_thermal_slowdown", "hw_slowdown"))])
    assert hot["reasons"] == ["hw_slowdown", "hw_thermal_slowdown"]


def test_traffic_follows_the_smoother_source(tmp_path, monkeypatch):
    src = tmp_path / "kernels.cuh"
    shutil.copy(bench.KERNEL_SRC, src)
    monkeypatch.setattr(bench, "KERNEL_SRC", str(src))
    text = src.read_text()
    assert MARK in text
    h0 = bench.kernel_hash()
    assert len(h0) == 16 and int(h0, 16) >= 0

    prof = tmp_path / "profile.txt"
    prof.write_text("# summary\nkernel_source_sha256_16 = %s\ndram_bytes_per_launch = 37763072\n" % h0)
    monkeypatch.setattr(bench, "TRAFFIC_FILE", str(prof))
    assert bench.measured_traffic() == 37763072.0

    # an edit after the transfer kernels' marker keeps the recorded traffic
    src.write_text(text + "\n// a later kernel\n")
    assert bench.kernel_hash() == h0 and bench.measured_traffic() == 37763072.0
    # an edit in the smoother's part drops it
    i = text.index(MARK)
    src.write_text(text[:i] + "// changed\n" + text[i:])
    assert bench.kernel_hash() != h0 and bench.measured_traffic() is None
    # a missing summary reports nothing rather than failing
    monkeypatch.setattr(bench, "TRAFFIC_FILE", str(tmp_path / "absent.txt"))
    assert bench.measured_traffic() is None


def test_committed_profile_names_a_hash_and_bytes():
    vals = {}
    with open(os.path.join(os.path.dirname(bench.__file__), "profiles", "k_smooth_spinodal512.txt")) as f:
        for line in f:
            if "=" in line and not line.startswith("#"):
                k, v = line.split("=", 1)
                vals[k.strip()] = v.strip()
    assert len(vals["kernel_source_sha256_16"]) == 16
    assert float(vals["dram_bytes_per_launch"]) > 0


def test_l2_roofline_fields():
    # algorithmic and request bytes per launch over the duration, against the probe's bandwidth
    r = bench.l2_roofline(1e7, 1e-5, 2e4, 2e7, "why")
    assert r["algorithmic_gbs"] == pytest.approx(1000.0) and r["frac_algorithmic"] == pytest.approx(0.05)
    assert r["achieved_gbs"] == pytest.approx(2000.0) and r["frac"] == pytest.approx(0.1)
    assert r["traffic"] == 2e7 and r["note"] == "why"
    # no request bytes recorded: no achieved figure; no probe: no fractions at all
    assert "achieved_gbs" not in bench.l2_roofline(1e7, 1e-5, 2e4, None, "why")
    assert bench.l2_roofline(1e7, 1e-5, None, 2e7, "why")["peak_gbs"] is None


def test_committed_3d_profiles_match_the_3d_source():
    # the 3D pass's summaries were taken on the current colour-pass source and name their bytes
    src = bench.KERNEL_SRC_3D
    assert bench.measured_traffic(bench.TRAFFIC_FILE_3D, src) > 0
    assert bench.measured_traffic(bench.TRAFFIC_FILE_3D, src, "l2_request_bytes_per_launch") > 0
    assert bench.measured_traffic(bench.TRAFFIC_FILE_256, src) > 0
    assert bench.measured_traffic(key="l2_request_bytes_per_launch") > 0
    assert bench.measured_traffic(bench.TRAFFIC_FILE_3D, src, "no_such_key") is None
