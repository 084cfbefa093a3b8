"""bench.py's host-side arithmetic, checked on the CPU: the clock summary
parsed from nvidia-smi samples (median SM clock under load, the throttle
reasons that were active), the whole-step roofline, and the peak it divides
by (the measured copy bandwidth, else the stated fallback)."""
import json
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402


def _sampler(lines):
    s = bench.ClockSampler(0)
    s.lines = list(lines)
    return s


def test_clock_summary_median_and_reasons():
    # index, sm, max sm, power, active mask, hw_slowdown, hw_thermal, sw_thermal, sw_power_cap
    lines = ["0, 2070, 2070, 900.1, 0x0, Not Active, Not Active, Not Active, Not Active",
             "0, 1980, 2070, 1390.0, 0x4, Not Active, Not Active, Not Active, Active",
             "0, 2070, 2070, 1100.5, 0x0, Not Active, Not Active, Not Active, Not Active"]
    s = _sampler(lines).summary()
    assert s["sm_mhz"] == 2070 and s["sm_max_mhz"] == 2070 and s["samples"] == 3
    assert s["reasons"] == ["sw_power_cap"] and not s["below_max_without_reason"]


def test_clock_summary_flags_every_slowdown_kind():
    lines = ["0, 1500, 2070, 1400, 0x88, Active, Active, Active, Not Active"]
    s = _sampler(lines).summary()
    assert s["reasons"] == ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown"]
    assert s["sm_mhz"] == 1500


def test_clock_summary_flags_a_clock_lock():
    lines = ["0, 1200, 2070, 600, 0x0, Not Active, Not Active, Not Active, Not Active"] * 5
    assert _sampler(lines).summary()["below_max_without_reason"]


def test_clock_summary_skips_malformed_samples():
    lines = ["", "0, [N/A], 2070, 1, 0x0, Not Active, Not Active, Not Active, Not Active",
             "garbage", "0, 1965, 2070, 1000, 0x0, Not Active, Not Active, Not Active, Not Active"]
    s = _sampler(lines).summary()
    assert s["samples"] == 1 and s["sm_mhz"] == 1965 and s["reasons"] == []
    assert not s["below_max_without_reason"]
    assert _sampler([]).summary() == {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unavailable"]}


def test_step_roofline_arithmetic():
    peak, kind = bench.measured_peak()
    r = bench.step_roofline(32800.0)  # MLUPS
    assert r["bound"] == "hbm" and r["unit"] == "GB/s" and r["bytes_per_site"] == 80
    assert r["achieved"] == pytest.approx(32800e6 * 80 / 1e9)
    assert r["frac"] == pytest.approx(r["achieved"] / peak)
    assert r["peak"] == peak and r["peak_kind"] == kind


def test_measured_peak_file_and_fallback(tmp_path, monkeypatch):
    (tmp_path / "MEASURED_PEAKS.json").write_text(json.dumps({"hbm_gbs": 6786.6, "bf16_tflops": 1914.3}))
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    assert bench.measured_peak() == (6786.6, "measured")
    os.remove(tmp_path / "MEASURED_PEAKS.json")
    assert bench.measured_peak() == (6800.0, "fallback")
