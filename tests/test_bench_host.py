"""Host logic of the benchmark on CPU: the clock sampler's parsing of nvidia-smi lines (median SM
clock, throttle reasons), the peak table, and the profile lookup for roofline traffic."""
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


def test_clock_sampler_parses_median_and_reasons():
    cs = bench.ClockSampler(0)
    cs.lines = [
        "0, 2070, 2070, 900.5, 0x0000000000000000, Not Active, Not Active, Not Active, Not Active",
        "0, 1980, 2070, 1350.0, 0x0000000000000004, Not Active, Not Active, Not Active, Active",
        "0, 2070, 2070, 1000.0, 0x0000000000000000, Not Active, Not Active, Not Active, Not Active",
        "0, [N/A], 2070, 1000.0, 0x0, Not Active, Not Active, Not Active, Not Active",
        "garbage",
    ]
    d = cs.stop()
    assert d == {"sm_mhz": 2070.0, "sm_max_mhz": 2070.0, "reasons": ["sw_power_cap"], "samples": 3}


def test_clock_sampler_flags_thermal_slowdown():
    cs = bench.ClockSampler(0)
    cs.lines = ["0, 1200, 2070, 1400.0, 0x48, Active, Active, Not Active, Not Active"]
    assert cs.stop()["reasons"] == ["hw_slowdown", "hw_thermal_slowdown"]


def test_peaks_and_profile_lookup():
    peaks, kind = bench.load_peaks()
    assert kind in ("measured", "fallback")
    assert peaks["bf16_tflops"] > 1000 and peaks["hbm_gbs"] > 1000
    traffic, src = bench.profiled_traffic("no_such_workload", "f16x3")
    assert traffic is None and src is None
    traffic, src = bench.profiled_traffic("si64_g96", "f16x3")
    if traffic is not None:  # None once the kernel source has changed since the counters were taken
        assert traffic > 0 and src.startswith("profiles" + os.sep)
