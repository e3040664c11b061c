"""Host logic of bench.py that needs no GPU: the per-form kernel classes and
roofline fractions, the clock/throttle summary the
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


class _FakeProfile:
    """Stands in for a handle's profile_read: kind -> (ms, launches, flops)."""

    def __init__(self, table):
        self.table = table

    def profile_read(self, kind):
        ms, n, fl = self.table.get(kind, (0.0, 0, 0.0))
        return {"ms": ms, "launches": n, "flops": fl}


def test_kernel_classes_of_each_precision_form():
    """Class records and roofline fractions from profiled times: executed flops
    credit 6 products for BF16x6 and 28 digit-plane products for the
    FP64-accurate form, against the BF16 peak; the FP64 path against the FP64
    GEMM rate."""
    import bench
    peaks = {"bf16_tflops_sustained": 1000.0, "hbm_gbs": 5000.0}
    # BF16x6: 10 ms of wide products with 1e12 algorithmic flops -> 6e12 executed -> 600 TFLOP/s
    g = _FakeProfile({5: (10.0, 4, 1e12), 7: (2.0, 8, 5e9), 8: (1.0, 8, 1e9), 2: (1.0, 10, 1e9), 1: (3.0, 2, 4.0)})
    cl = bench.kernel_classes(g, "bf16x6", 20.0, 1, peaks, "test", 1.0)
    wide = cl[0]
    assert wide["bound"] == "tensor" and abs(wide["achieved"] - 600.0) < 1e-9 and abs(wide["frac"] - 0.6) < 1e-12
    assert cl[1]["bound"] == "hbm" and abs(cl[1]["achieved"] - 2500.0) < 1e-9
    assert any(c["bound"] == "latency" for c in cl) and cl[-1]["mean_sweeps_per_call"] == 4.0
    # FP64-accurate: 100 ms of products with 1e12 algorithmic flops -> 28e12 executed -> 280 TFLOP/s
    g = _FakeProfile({0: (100.0, 50, 1e12), 2: (5.0, 20, 1e9), 1: (4.0, 2, 7.0)})
    cl = bench.kernel_classes(g, "fp64tc", 200.0, 1, peaks, "test", 1.0)
    assert cl[0]["bound"] == "tensor" and abs(cl[0]["achieved"] - 280.0) < 1e-9
    assert abs(cl[0]["fp64_equivalent_tflops"] - 10.0) < 1e-9 and abs(cl[0]["frac"] - 0.28) < 1e-12
    # FP64: the CUDA-core GEMM class against the FP64 rate
    g = _FakeProfile({0: (1000.0, 50, 1e12), 1: (4.0, 2, 7.0)})
    cl = bench.kernel_classes(g, "fp64", 2000.0, 1, peaks, "test", 1.1)
    assert cl[0]["bound"] == "alu" and abs(cl[0]["frac"] - 1.0 / 1.1) < 1e-12
    assert not any(c["bound"] == "latency" for c in cl)
