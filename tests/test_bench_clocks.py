"""The clock record of bench.py: NVML reason bits and nvidia-smi rows become the named
throttle reasons a bench line reports (hw_slowdown, hw_thermal_slowdown, sw_thermal_slowdown,
sw_power_cap), the denser NVML samples give the median clock when present, and a host with
neither tool says so instead of reporting a clock."""
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


def test_nvml_bits_name_the_reasons():
    # bits of nvml.h: 0x4 SwPowerCap, 0x8 HwSlowdown, 0x20 SwThermalSlowdown, 0x40 HwThermalSlowdown;
    # 0x1 (GpuIdle) and 0x2 (ApplicationsClocksSetting) are not reasons the record names
    cases = {0x0: [], 0x1: [], 0x2: [], 0x4: ["sw_power_cap"], 0x8: ["hw_slowdown"],
             0x20: ["sw_thermal_slowdown"], 0x40: ["hw_thermal_slowdown"],
             0x4 | 0x40: ["hw_thermal_slowdown", "sw_power_cap"]}
    for bits, want in cases.items():
        rec = bench.summarise_clocks([(2070, 2070, bits)], [])
        assert rec["reasons"] == sorted(want), hex(bits)


def test_median_and_source():
    nv = [(2070, 2070, 0), (1980, 2070, 0x4), (2070, 2070, None)]
    rec = bench.summarise_clocks(nv, [])
    assert rec["sm_mhz"] == 2070.0 and rec["sm_max_mhz"] == 2070.0
    assert rec["samples"] == 3 and rec["source"] == "nvml"
    assert rec["reasons"] == ["sw_power_cap"]


def test_nvidia_smi_rows():
    rows = ["1965, 2070, 1100.5, 0x0000000000000004, Not Active, Not Active, Not Active, Active",
            "2070, 2070, 1200.0, 0x0000000000000000, Not Active, Not Active, Not Active, Not Active",
            "garbage line",
            "[N/A], 2070, 1.0, 0x0, Not Active, Not Active, Not Active, Not Active"]
    rec = bench.summarise_clocks([], rows)
    assert rec["source"] == "nvidia-smi" and rec["samples"] == 2 and rec["nvidia_smi_samples"] == 2
    assert rec["sm_mhz"] == (1965 + 2070) / 2 and rec["reasons"] == ["sw_power_cap"]
    # a hardware slowdown seen only by nvidia-smi still reaches the record when NVML gave the clocks
    hot = ["2070, 2070, 900.0, 0x8, Active, Not Active, Not Active, Not Active"]
    rec = bench.summarise_clocks([(2070, 2070, 0)], hot)
    assert rec["source"] == "nvml" and rec["reasons"] == ["hw_slowdown"]


def test_no_tool_no_clock():
    rec = bench.summarise_clocks([], [])
    assert rec["sm_mhz"] is None and rec["samples"] == 0 and rec["source"] is None


def test_sampler_on_a_host_without_a_gpu():
    # neither libnvidia-ml nor nvidia-smi need exist here; the sampler must still return a record
    s = bench.ClockSampler(0)
    s.start()
    rec = s.stop()
    assert set(rec) >= {"sm_mhz", "sm_max_mhz", "reasons", "samples"}
    if rec["samples"] == 0:
        assert rec["sm_mhz"] is None


class _FakeNVML:
    """Stands in for libnvidia-ml: answers the read-only queries the sampler makes."""

    def __init__(self, uuid_ok):
        self.uuid_ok = uuid_ok
        self.calls = []
        self.open = 0

    def nvmlInit_v2(self):
        self.open += 1
        return 0

    def nvmlShutdown(self):
        self.open -= 1
        return 0

    def nvmlDeviceGetHandleByUUID(self, u, h):
        self.calls.append(("uuid", u))
        if not self.uuid_ok:
            return 13
        h._obj.value = 0x1000
        return 0

    def nvmlDeviceGetHandleByIndex_v2(self, i, h):
        self.calls.append(("index", i.value))
        h._obj.value = 0x2000
        return 0

    def nvmlDeviceGetClockInfo(self, h, kind, out):
        assert kind == 1  # the SM clock domain
        out._obj.value = 1995
        return 0

    def nvmlDeviceGetMaxClockInfo(self, h, kind, out):
        out._obj.value = 2070
        return 0

    def nvmlDeviceGetCurrentClocksEventReasons(self, h, out):
        out._obj.value = 0x4
        return 0


def test_sampler_with_a_fake_nvml(monkeypatch):
    import ctypes
    import time
    for uuid_ok in (True, False):
        fake = _FakeNVML(uuid_ok)
        monkeypatch.setattr(ctypes, "CDLL", lambda name: fake)
        monkeypatch.setattr(bench.subprocess, "Popen", lambda *a, **k: (_ for _ in ()).throw(OSError("none")))
        s = bench.ClockSampler(3, "0fa0a3b8-1111-2222-3333-444455556666")
        s.start()
        time.sleep(0.05)
        rec = s.stop()
        assert rec["source"] == "nvml" and rec["samples"] >= 3
        assert rec["sm_mhz"] == 1995.0 and rec["sm_max_mhz"] == 2070.0 and rec["reasons"] == ["sw_power_cap"]
        assert fake.calls[0] == ("uuid", b"GPU-0fa0a3b8-1111-2222-3333-444455556666")
        assert (("index", 3) in fake.calls) == (not uuid_ok)
        assert fake.open == 0  # shut down again
