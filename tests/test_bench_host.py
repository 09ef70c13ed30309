"""Host logic of bench.py that needs no GPU: clock-sample parsing over the timed region, the censored median of
time-to-target runs, and the description of the host the CPU oracle runs on."""

import datetime
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


def _line(t, sm, mx=2070, reasons=("Not Active",) * 4):
    stamp = datetime.datetime.fromtimestamp(t).strftime("%Y/%m/%d %H:%M:%S.%f")[:-3]
    return ", ".join([stamp, "0", str(sm), str(mx), "900.00", "0x0"] + list(reasons)) + "\n"


def test_clock_samples_inside_the_timed_region():
    t0 = 1_800_000_000.0
    lines = [_line(t0 - 1.0, 345), _line(t0 + 0.1, 2070), _line(t0 + 0.2, 1995), _line(t0 + 0.3, 2070),
             _line(t0 + 2.0, 345), "not a sample\n"]
    out = bench.parse_clock_samples(lines, t0, t0 + 0.35)
    assert out["samples"] == 3 and out["in_timed_region"]
    assert out["sm_mhz"] == 2070 and out["sm_max_mhz"] == 2070 and out["reasons"] == []


def test_clock_samples_report_throttle_reasons_and_fall_back_when_none_inside():
    t0 = 1_800_000_000.0
    hot = ("Not Active", "Active", "Not Active", "Active")  # hw_thermal_slowdown and sw_power_cap
    lines = [_line(t0 - 5.0, 1500, reasons=hot), _line(t0 - 4.9, 1600)]
    out = bench.parse_clock_samples(lines, t0, t0 + 0.01)
    assert not out["in_timed_region"] and out["samples"] == 2
    assert out["reasons"] == ["hw_thermal_slowdown", "sw_power_cap"]
    assert out["sm_mhz"] == 1550


def test_censored_median():
    assert bench.censored_median([3.0, 1.0, 2.0]) == 2.0
    assert bench.censored_median([None, 1.0, 2.0, 4.0, None]) == 4.0  # two runs never reached the target
    assert bench.censored_median([None, 1.0, None]) is None  # most runs never reached it
    assert bench.censored_median([1.0, 3.0]) == 2.0
    assert bench.censored_median([1.0, None]) is None
    assert bench.censored_median([]) is None


def test_host_description_names_the_cores():
    h = bench.host_description()
    assert h["cores"] >= 1 and h["machine"]


def test_issue_roofline_from_the_committed_profiles():
    """The instruction-issue peak is the unit count times the clock; the profiles' instruction counts give a fraction
    below 1 at the measured launch times (skipped when the profiles predate the kernel source)."""
    import pytest

    assert bench.ISSUE_PEAK == 152 * 4 * 2.07e9
    none = bench.issue_roofline("no_such_workload", 1.0)
    assert none["bound"] == "alu" and none["achieved"] is None and none["frac"] is None
    r = bench.issue_roofline("euclid10000_p100", 1.142)
    if r["achieved"] is None:
        pytest.skip("profiles were taken on another kernel source")
    assert 0.3 < r["frac"] < 1.0 and r["bound"] == "alu"
    assert r["achieved"] == pytest.approx(r["instructions_per_launch"] / 1.142e-3)


def test_golden_optimum_reader():
    cost, best = bench.golden_optimum("graph100")
    assert cost == 5747 and best == (5, 17, 40, 42, 57)
