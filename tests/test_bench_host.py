"""Host logic of bench.py that the JSON line depends on (no GPU): the clock
record taken during the timed region and the roofline's peak."""
import importlib.util
import json
import os

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def bench():
    spec = importlib.util.spec_from_file_location("bench", os.path.join(ROOT, "bench.py"))
    m = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(m)
    return m


def _row(mhz, watts, reasons=("Not Active",) * 4):
    return ", ".join(["0", str(mhz), "2070", str(watts), "0x0"] + list(reasons))


def test_clock_summary_takes_the_loaded_samples(bench):
    c = bench.Clocks(0)
    c.out = "\n".join([_row(1200, 150), _row(2070, 900), _row(2070, 950),
                       _row(2055, 980, ("Not Active", "Not Active", "Not Active", "Active")),
                       "garbage line", _row(1100, 140)])
    s = c.summary()
    # idle samples (power below 30% of the maximum) are left out of the median
    assert s["sm_mhz"] == 2070 and s["sm_max_mhz"] == 2070 and s["samples"] == 5
    assert s["reasons"] == ["sw_power_cap"]


def test_clock_summary_reports_thermal_and_missing_samples(bench):
    c = bench.Clocks(0)
    c.out = _row(1800, 1000, ("Not Active", "Active", "Not Active", "Not Active"))
    assert c.summary()["reasons"] == ["hw_thermal_slowdown"]
    c.out = ""
    assert c.summary() == {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unavailable"], "samples": 0}


def test_peak_is_the_measured_copy_bandwidth(bench):
    peak, kind = bench._peaks()
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        assert kind == "measured" and peak == float(json.load(open(path))["hbm_gbs"])
    else:
        assert kind == "fallback" and peak == 6800.0
