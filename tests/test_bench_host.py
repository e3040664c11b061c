"""Host logic of bench.py that needs no GPU: the clock/throttle summary the
bench line carries (nvidia-smi CSV rows as the sampler receives them) and the
roofline denominators' source."""
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


def _sampler(lines):
    s = bench.ClockSampler(0)
    s.lines = list(lines)
    return s


def test_clock_summary_median_max_and_active_reasons():
    rows = [
        "0, 2070, 2070, 650.1, 0x0000000000000000, Not Active, Not Active, Not Active, Not Active",
        "0, 2055, 2070, 990.4, 0x0000000000000004, Not Active, Not Active, Not Active, Active",
        "0, 1980, 2070, 1390.0, 0x0000000000000004, Not Active, Not Active, Not Active, Active",
        "garbage line",
        "0, [N/A], 2070, 1.0, 0x0, Not Active, Not Active, Not Active, Not Active",
    ]
    out = _sampler(rows).summary()
    assert out["sm_mhz"] == 2055.0 and out["sm_max_mhz"] == 2070.0
    assert out["reasons"] == ["sw_power_cap"] and out["samples"] == 3


def test_clock_summary_flags_thermal_and_unsampled():
    rows = ["0, 1500, 2070, 1400.0, 0x48, Active, Not Active, Active, Not Active"]
    out = _sampler(rows).summary()
    assert out["reasons"] == ["hw_slowdown", "sw_thermal_slowdown"]
    assert _sampler([]).summary() == {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}


def test_peaks_come_from_the_measured_file_when_present():
    peaks, source = bench.measured_peaks()
    if os.path.exists(os.path.join(ROOT, "MEASURED_PEAKS.json")):
        assert source == "measured"
    else:
        assert source == "fallback" and peaks["hbm_gbs"] == 6800.0
    assert peaks
