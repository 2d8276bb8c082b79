"""Host logic of bench.py: the clock sampler's filtering to the timed region and decoding
of NVML clock-event reasons, the CPU baseline's JSON fields, and the TTS formula (Eq. 9)
against the oracle's."""
import math

import pytest

import bench
import oracle as o


def test_clock_sampler_keeps_only_samples_inside_the_region():
    cs = bench.ClockSampler(0)
    cs.source = "nvml, 5 ms"
    cs.t0, cs.t1 = 100.0, 100.010
    cs.lines = [
        "99.999000,1200,2070,1",            # before the region: dropped
        "100.001000,2070,2070,0",
        "100.004000,2055,2070,4",           # sw_power_cap
        "100.007000,2070,2070,72",          # hw_slowdown | hw_thermal_slowdown
        "100.011000,300,2070,32",           # after the region: dropped
        "garbage",
    ]
    s = cs.summary()
    assert s["samples"] == 3 and s["sm_mhz"] == 2070.0 and s["sm_max_mhz"] == 2070.0
    assert s["sm_mhz_min"] == 2055.0
    assert s["reasons"] == ["hw_slowdown", "hw_thermal_slowdown", "sw_power_cap"]


def test_clock_sampler_nvidia_smi_lines():
    cs = bench.ClockSampler(0)
    cs.source = "nvidia-smi, 200 ms"
    cs.t0, cs.t1 = 0.0, 1.0
    cs.lines = ["0, 1965, 2070, 900.1, 0x4, Not Active, Not Active, Not Active, Active"]
    s = cs.summary()
    assert s["samples"] == 1 and s["sm_mhz"] == 1965.0 and s["reasons"] == ["sw_power_cap"]


def test_clock_sampler_without_samples():
    cs = bench.ClockSampler(0)
    cs.t0, cs.t1 = 0.0, 1.0
    s = cs.summary()
    assert s["samples"] == 0 and s["sm_mhz"] is None


def test_cpu_baseline_fields():
    r = bench.cpu_baseline(bench.WORKLOADS["dense200"], sample_replicas=4)
    assert r["kind"] == "oracle" and r["unit"] == bench.METRIC and r["cores"] >= 1
    assert r["value"] > 0 and "4 of the 1024 replicas" in r["sample"] and "extrapolated" in r["sample"]
    w = dict(bench.WORKLOADS["sk16"])
    r = bench.cpu_baseline(w)      # the whole workload: nothing extrapolated
    assert "1 of the 1 replicas x 1000 of 1000" in r["sample"] and "extrapolated" not in r["sample"]


def test_default_workload_is_the_largest_single_gpu_configuration():
    w = bench.WORKLOAD
    assert (w["N"], w["replicas"], w["iterations"]) == (2000, 4096, 5000)
    assert w["cpu_replicas"] * w["cpu_iters"] < w["replicas"] * w["iterations"]


@pytest.mark.parametrize("t1,p", [(2.0, 0.9), (1.0, 0.5), (3e-6, 0.074), (1.0, 0.99), (1.0, 1.0), (1.0, 0.0),
                                  (1.0, 1e-4)])
def test_tts99_matches_the_oracle(t1, p):
    a, b = bench.tts99(t1, p), o.tts(t1, p)
    assert (math.isinf(a) and math.isinf(b)) or a == pytest.approx(b, rel=1e-12)
