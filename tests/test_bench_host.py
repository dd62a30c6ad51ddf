"""Host logic of bench.py that needs no GPU: the key under which stored ncu
traffic figures stay attached to a kernel's code, and the summary of the
clock and throttle samples taken during the timed region."""
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402

SRC = """// a kernel
__global__ void k(float *x) {   /* one
   block */
    x[threadIdx.x] *= 2.f;      // doubled
}
"""


def test_code_hash_ignores_comments_and_blank_space():
    h = bench.code_sha256(SRC)
    edited = SRC.replace("// doubled", "// twice its value").replace("/* one\n   block */", "")
    assert bench.code_sha256(edited) == h
    assert bench.code_sha256(SRC.replace("    x[", "\tx[")) == h


def test_code_hash_changes_with_the_code():
    h = bench.code_sha256(SRC)
    assert bench.code_sha256(SRC.replace("2.f", "3.f")) != h
    assert bench.code_sha256(SRC.replace("threadIdx.x]", "threadIdx.x + 1]")) != h


def test_stored_traffic_needs_a_matching_entry():
    assert bench.stored_traffic("induced_current.cu", "no_such_workload") is None


def _line(sm, mx, power, reasons=()):
    names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
    flags = ["Active" if n in reasons else "Not Active" for n in names]
    return ", ".join(["0", str(sm), str(mx), str(power), "0x0000000000000000"] + flags)


def test_clock_summary_median_max_and_reasons():
    lines = [_line(2070, 2070, 310.5), _line(2040, 2070, 690.0, {"sw_power_cap"}), _line(2070, 2070, 420.0)]
    s = bench.ClockSampler.summarize(lines)
    assert s["sm_mhz"] == 2070.0 and s["sm_max_mhz"] == 2070.0 and s["samples"] == 3
    assert s["power_w_max"] == 690.0
    assert s["reasons"] == ["sw_power_cap"]


def test_clock_summary_keeps_reasons_of_samples_whose_numbers_do_not_parse():
    lines = [_line(1500, 2070, "[N/A]", {"hw_thermal_slowdown"}), _line("[N/A]", "[N/A]", "[N/A]", {"hw_slowdown"}),
             "garbage", ""]
    s = bench.ClockSampler.summarize(lines)
    assert s["sm_mhz"] == 1500.0 and s["samples"] == 1 and s["power_w_max"] is None
    assert s["reasons"] == ["hw_slowdown", "hw_thermal_slowdown"]
    assert bench.ClockSampler.summarize([])["reasons"] == ["no samples"]
