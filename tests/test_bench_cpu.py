"""The benchmark's host-side bookkeeping on CPU: the clock record taken during the timed region
(median SM clock, maximum, throttle reasons marked Active) and the measured HBM peak read from
the peaks file, whatever its nesting."""
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


def _sampler(lines):
    s = bench.ClockSampler()
    s.lines = list(lines)
    return s


def test_clock_summary_median_max_and_reasons():
    lines = ["0, 2070, 2070, 1100.5, 0x0000000000000000, Not Active, Not Active, Not Active, Not Active",
             "0, 1980, 2070, 1390.2, 0x0000000000000004, Not Active, Not Active, Not Active, Active",
             "0, 2010, 2070, 1380.0, 0x0000000000000004, Not Active, Not Active, Not Active, Active",
             "garbage line",
             "0, [N/A], 2070, [N/A], [N/A], [N/A], [N/A], [N/A], [N/A]"]
    s = _sampler(lines).summary()
    assert s["sm_mhz"] == 2010.0 and s["sm_max_mhz"] == 2070.0 and s["samples"] == 3
    assert s["reasons"] == ["sw_power_cap"]


def test_clock_summary_flags_slowdowns():
    lines = ["0, 1200, 2070, 900.0, 0x08, Active, Not Active, Not Active, Not Active",
             "0, 1100, 2070, 900.0, 0x48, Active, Active, Active, Not Active"]
    s = _sampler(lines).summary()
    assert s["reasons"] == ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown"]
    assert s["sm_mhz"] == 1150.0


def test_clock_summary_without_samples():
    s = _sampler([]).summary()
    assert s["sm_mhz"] is None and s["samples"] == 0 and s["reasons"] == []


def test_hbm_peak_from_the_peaks_file_layouts():
    assert bench.hbm_peak_gbs({"hbm_gbs": 6683.5, "bf16_tflops": 1963.2}) == 6683.5
    assert bench.hbm_peak_gbs({"gpu": {"gbs": 7000.0}}) == 7000.0
    assert bench.hbm_peak_gbs({"bf16_tflops": 1900.0}) == 6800.0          # the stated fallback
    d, kind = bench.peaks()
    assert kind in ("measured", "fallback") and bench.hbm_peak_gbs(d) > 1000.0
