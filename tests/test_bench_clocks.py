"""The bench's clock record keeps the samples taken inside the timed region.

A fake nvidia-smi (a Python script printing the same CSV fields, timestamp first) and a
fake NVML (the calls the NVML sampler makes) stand in for the real ones, so this runs on
the CPU."""

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


class FakeNvml:
    """Stands in for libnvidia-ml: the calls the NVML sampler makes, by ctypes convention
    (results written through byref arguments, 0 = success)."""

    def __init__(self, reasons=0x4, init_rc=0):
        self.n = 0
        self.reason_bits = reasons
        self.init_rc = init_rc
        self.shut = False

    def nvmlInit_v2(self):
        return self.init_rc

    def nvmlShutdown(self):
        self.shut = True
        return 0

    def nvmlDeviceGetHandleByPciBusId_v2(self, bus, h):
        h._obj.value = 1
        return 0

    def nvmlDeviceGetHandleByIndex_v2(self, i, h):
        h._obj.value = 1
        return 0

    def nvmlDeviceGetMaxClockInfo(self, h, kind, out):
        out._obj.value = 2070
        return 0

    def nvmlDeviceGetClockInfo(self, h, kind, out):
        assert kind == 1   # the SM clock
        out._obj.value = 1965 if self.n % 2 else 1995
        self.n += 1
        return 0

    def nvmlDeviceGetCurrentClocksEventReasons(self, h, out):
        out._obj.value = self.reason_bits
        return 0


def test_nvml_samples_inside_the_window():
    nv = FakeNvml()
    with bench.NvmlClockSampler(0, interval_ms=5, lib=nv) as clk:
        assert clk.ok
        time.sleep(0.05)                 # samples before the region are dropped
        clk.start()
        time.sleep(0.2)
        clk.stop()
    s = clk.summary()
    assert 15 <= s["samples"] <= 60, s
    assert s["sm_mhz"] in (1965.0, 1980.0, 1995.0) and s["sm_max_mhz"] == 2070.0
    assert s["reasons"] == ["sw_power_cap"] and s["source"] == "nvml"
    assert all(clk.t0 <= r[0] <= clk.t1 for r in clk.window())
    assert nv.shut


def test_nvml_reason_bits_map_to_names():
    with bench.NvmlClockSampler(0, interval_ms=5, lib=FakeNvml(reasons=0x8 | 0x40 | 0x1)) as clk:
        clk.start()
        time.sleep(0.03)
        clk.stop()
    assert clk.summary()["reasons"] == ["hw_slowdown", "hw_thermal_slowdown"]


def test_nvml_failure_is_reported_not_raised():
    with bench.NvmlClockSampler(0, lib=FakeNvml(init_rc=1)) as clk:
        assert not clk.ok
        clk.start()
        clk.stop()
    assert clk.summary()["samples"] == 0


def test_sampler_falls_back_to_nvidia_smi_without_nvml(monkeypatch):
    class NoNvml(bench.NvmlClockSampler):
        def __init__(self, device):
            super().__init__(device, lib=FakeNvml(init_rc=1))
    monkeypatch.setattr(bench, "NvmlClockSampler", NoNvml)
    monkeypatch.setattr(bench.ClockSampler, "_command", lambda self, ms: [sys.executable, "-c", "pass"])
    with bench.clock_sampler(0) as clk:
        assert isinstance(clk, bench.ClockSampler)
        clk.start()
        clk.stop()
    assert clk.summary()["source"] == "nvidia-smi"
