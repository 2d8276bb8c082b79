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


def _tts_args(**kw):
    import argparse
    a = dict(tts_jump=0.0, tts_eps=0.0, tts_gamma=0.0, tts_refresh=0)
    a.update(kw)
    return argparse.Namespace(**a)


def test_tts_family_schedule_and_the_heuristic():
    from paper_2407_10205_gb300 import instances as ins, schedules
    w = bench.WORKLOADS["tts"]
    d3 = ins.family_instance("maxcut_d3", 64, 3)
    sk = ins.family_instance("sk_ising", 64, 3)
    own = bench.tts_schedule_params(w, _tts_args(), "maxcut_d3", d3)
    f = w["family_schedule"]["maxcut_d3"]
    assert own[2:] == (f["eps"], f["gamma"], f["refresh"])
    assert own[1] == pytest.approx(f["jump"] / schedules.field_scale(d3)) and own[0] == pytest.approx(own[1] / 20)
    # the reference's second run: the heuristic alone, default final jump for n = 64
    assert bench.tts_schedule_params(w, _tts_args(), "maxcut_d3", d3, own=False) == schedules.suggest_schedule(d3)
    # a family without an entry runs the heuristic
    assert bench.tts_schedule_params(w, _tts_args(), "sk_ising", sk) == schedules.suggest_schedule(sk)
    # command-line values win over the family's
    o = bench.tts_schedule_params(w, _tts_args(tts_eps=0.05, tts_refresh=7, tts_jump=3.0), "maxcut_d3", d3)
    assert o[2:] == (0.05, f["gamma"], 7) and o[1] == pytest.approx(3.0 / schedules.field_scale(d3))
