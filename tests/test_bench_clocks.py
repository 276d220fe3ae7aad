"""The bench's clock record keeps the nvidia-smi samples taken inside the timed region.

A fake nvidia-smi (a Python script printing the same CSV fields, timestamp first) stands
in for the real one, so this runs on the CPU."""

import sys
import textwrap
import time

import pytest

import bench

FAKE = textwrap.dedent("""
    import datetime, sys, time
    period = float(sys.argv[1])
    for n in range(2000):
        ts = datetime.datetime.now().strftime("%Y/%m/%d %H:%M:%S.%f")[:-3]
        sm = 1965 if n % 2 else 1995
        print(f"{ts}, 0, {sm}, 2070, 912.5, 0x0000000000000004, Not Active, Not Active, Not Active, Active",
              flush=True)
        time.sleep(period)
""")


@pytest.fixture
def fake(tmp_path):
    p = tmp_path / "fake_smi.py"
    p.write_text(FAKE)
    return lambda period: [sys.executable, str(p), str(period)]


def test_samples_inside_the_window(fake):
    with bench.ClockSampler(0, interval_ms=20, cmd=fake(0.02)) as clk:
        time.sleep(0.1)                  # samples before the region are dropped
        clk.start()
        time.sleep(0.3)
        clk.stop()
        time.sleep(0.1)                  # and so are those after it
    s = clk.summary()
    assert 8 <= s["samples"] <= 20, s
    assert s["sm_mhz"] in (1965.0, 1980.0, 1995.0) and s["sm_max_mhz"] == 2070.0
    assert s["reasons"] == ["sw_power_cap"]
    assert 290 <= s["window_ms"] <= 400
    assert all(clk.t0 <= ts <= clk.t1 for ts, _ in clk.window())


def test_short_region_takes_the_next_sample(fake):
    with bench.ClockSampler(0, interval_ms=200, cmd=fake(0.2)) as clk:
        clk.start()
        clk.stop()                       # waits (bounded) for the first sample after the region
    s = clk.summary()
    assert s["samples"] == 1 and s["sm_mhz"] in (1965.0, 1995.0)
    assert clk.window()[0][0] >= clk.t0


def test_missing_tool_gives_an_empty_record():
    with bench.ClockSampler(0, cmd=[sys.executable, "-c", "pass"]) as clk:
        clk.start()
        clk.stop()
    s = clk.summary()
    assert s["samples"] == 0 and s["sm_mhz"] is None and s["reasons"] == []
