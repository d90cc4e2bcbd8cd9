"""bench.py's clock record: the median SM clock under load and the throttle
reasons seen while the timed region ran, parsed from nvidia-smi's CSV lines
(clocks.sm, clocks.max.sm, power.draw, active mask, then the four reasons)."""
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)


def _sampler(lines):
    import bench

    s = bench.ClockSampler(0)
    s.lines = list(lines)
    return s


def test_median_clock_and_no_reasons():
    s = _sampler(["2070, 2070, 900.1, 0x0000000000000000, Not Active, Not Active, Not Active, Not Active",
                  "1980, 2070, 1100.5, 0x0000000000000000, Not Active, Not Active, Not Active, Not Active",
                  "2055, 2070, 1010.0, 0x0000000000000000, Not Active, Not Active, Not Active, Not Active"])
    out = s.summary()
    assert out["sm_mhz"] == 2055.0 and out["sm_max_mhz"] == 2070.0
    assert out["reasons"] == [] and out["samples"] == 3


def test_reasons_are_collected_by_column():
    s = _sampler(["1800, 2070, 1390.0, 0x0000000000000004, Not Active, Not Active, Not Active, Active",
                  "1700, 2070, 1400.0, 0x0000000000000048, Not Active, Active, Not Active, Not Active",
                  "[N/A], 2070, [N/A], [N/A], [N/A], [N/A], [N/A], [N/A]",
                  "garbage"])
    out = s.summary()
    assert out["reasons"] == ["hw_thermal_slowdown", "sw_power_cap"]
    assert out["samples"] == 2 and out["sm_mhz"] == 1750.0


def test_no_samples_is_marked_unsampled():
    out = _sampler([]).summary()
    assert out["sm_mhz"] is None and out["reasons"] == ["unsampled"]
