"""Host logic of bench.py (CPU): the clock sampler keeps the samples stamped
inside the timed region, falls back to those taken right after a region too
short to hold any (saying so), reports the throttle reasons it saw, and uses
a line's arrival time when nvidia-smi's stamp cannot be read."""
import datetime
import importlib.util
import os

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def bench():
    spec = importlib.util.spec_from_file_location("bench_module", os.path.join(ROOT, "bench.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


def _line(t, sm=2070.0, active=(), stamp=True):
    ts = datetime.datetime.fromtimestamp(t).strftime("%Y/%m/%d %H:%M:%S.%f")[:-3]
    names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
    flags = ", ".join("Active" if n in active else "Not Active" for n in names)
    return (t, f"{ts if stamp else 'n/a'}, {sm}, 2070, 812.5, 0x0, {flags}")


def test_samples_inside_the_region(bench):
    t0 = 1_700_000_000.0
    lines = [_line(t0 - 0.5, 1200.0), _line(t0 + 0.1, 2070.0), _line(t0 + 0.2, 2040.0),
             _line(t0 + 0.3, 2055.0, ("sw_power_cap",)), _line(t0 + 0.9, 900.0)]
    c = bench.ClockSampler.summary(lines, t0, t0 + 0.35)
    assert c["samples"] == 3 and c["sm_mhz"] == 2055.0 and c["sm_max_mhz"] == 2070.0
    assert c["reasons"] == ["sw_power_cap"] and "window" not in c


def test_short_region_reports_the_samples_after_it(bench):
    t0 = 1_700_000_000.0
    lines = [_line(t0 - 0.05, 1000.0), _line(t0 + 0.06, 2070.0),
             _line(t0 + 0.11, 2070.0, ("hw_slowdown",))]
    c = bench.ClockSampler.summary(lines, t0, t0 + 0.04)
    assert c["samples"] == 0 and c["samples_after_region"] == 2
    assert c["reasons"] == ["hw_slowdown"] and "shorter than" in c["window"]


def test_unreadable_stamp_uses_the_arrival_time(bench):
    t0 = 1_700_000_000.0
    lines = [_line(t0 + 0.1, 2000.0, stamp=False), ("x", "garbage line")][:1]
    c = bench.ClockSampler.summary(lines, t0, t0 + 0.2)
    assert c["samples"] == 1 and c["sm_mhz"] == 2000.0


def test_no_samples_is_none(bench):
    assert bench.ClockSampler.summary([], 0.0, 1.0) is None
    s = bench.ClockSampler(0)
    assert s.need_more() is False  # not started: nothing to wait for
