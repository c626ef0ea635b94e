"""The clock record of bench.py, on CPU: NVML reads through a fake library
and the summary of NVML samples and nvidia-smi lines."""
import ctypes

import bench


class FakeNvml:
    """Answers the NVML calls the sampler makes; writes through the pointers."""

    def __init__(self, clock=1965, reasons=0x4 | 0x8, max_clock=2070, uuid_ok=True):
        self.clock, self.reasons, self.max_clock, self.uuid_ok = clock, reasons, max_clock, uuid_ok
        self.shut = False

    def nvmlInit_v2(self):
        return 0

    def nvmlShutdown(self):
        self.shut = True
        return 0

    def nvmlDeviceGetHandleByUUID(self, uuid, h):
        assert isinstance(uuid, bytes) and uuid.startswith(b"GPU-")
        return 0 if self.uuid_ok else 13

    def nvmlDeviceGetHandleByIndex_v2(self, index, h):
        return 0

    def nvmlDeviceGetClockInfo(self, h, kind, out):
        assert kind == 1   # the SM clock
        out._obj.value = self.clock
        return 0

    def nvmlDeviceGetMaxClockInfo(self, h, kind, out):
        out._obj.value = self.max_clock
        return 0

    def nvmlDeviceGetCurrentClocksEventReasons(self, h, out):
        out._obj.value = self.reasons
        return 0


def test_nvml_sample_decodes_clock_and_reasons():
    lib = FakeNvml()
    n = bench._Nvml("GPU-0000", 0, lib=lib)
    clock, reasons = n.sample()
    assert clock == 1965 and sorted(reasons) == ["hw_slowdown", "sw_power_cap"]
    assert n.max_sm() == 2070
    n.close()
    assert lib.shut
    # a UUID NVML does not know: the index is used instead
    n = bench._Nvml("GPU-ffff", 3, lib=FakeNvml(reasons=0, uuid_ok=False))
    assert n.sample() == (1965, [])


def test_summary_prefers_nvml_samples_and_merges_reasons():
    smi = ("0, 2070, 2070, 900.5, 0x0000000000000000, Not Active, Not Active, Not Active, Not Active\n"
           "0, 1800, 2070, 1390.1, 0x0000000000000004, Not Active, Not Active, Not Active, Active\n")
    nv = [(2070, []), (2070, []), (2055, ["sw_power_cap"]), (2070, [])]
    r = bench.clock_summary(nv, 2070, smi)
    assert r["sm_mhz"] == 2070.0 and r["sm_min_mhz"] == 2055.0 and r["sm_max_mhz"] == 2070.0
    assert r["reasons"] == ["sw_power_cap"] and r["samples"] == 4 and r["nvidia_smi_samples"] == 2
    assert r["source"].startswith("nvml")
    # nvidia-smi alone; a throttling reason it reports is kept
    smi2 = "0, 1500, 2070, 700.0, 0x40, Not Active, Active, Not Active, Not Active\n"
    r = bench.clock_summary([], None, smi2)
    assert r["sm_mhz"] == 1500.0 and r["reasons"] == ["hw_thermal_slowdown"] and r["source"].startswith("nvidia-smi")
    # nothing at all
    assert bench.clock_summary([], None, "")["sm_mhz"] is None
