"""CPU checks of the benchmark's host logic: the clock record and the bounded oracle samples.

The timed arms need a GPU; what they report beside the number does not: the median SM clock and
the throttle reasons read from nvidia-smi's CSV lines (a reason seen active in any sample is
reported, since such a run is rejected), and the deterministic series samples the oracle is timed
on (every k-th series of the workload, the uneven workload's sample capped by its scan cost).
"""
import argparse
import os
import sys

import numpy as np

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
import bench  # noqa: E402


class _FakeProc:
    def __init__(self, text):
        self.text, self.terminated = text, False

    def terminate(self):
        self.terminated = True

    def communicate(self, timeout=None):
        return self.text, ""


def _sampler(lines):
    s = bench.ClockSampler(0)
    s.proc = _FakeProc("\n".join(lines) + "\n")
    return s


def test_clock_record_median_and_reasons():
    # fields: index, clocks.sm, clocks.max.sm, power.draw, active mask, hw_slowdown,
    # hw_thermal_slowdown, sw_thermal_slowdown, sw_power_cap
    lines = [
        "0, 2032, 2032, 640.1, 0x0000000000000000, Not Active, Not Active, Not Active, Not Active",
        "0, 1980, 2032, 1099.0, 0x0000000000000004, Not Active, Not Active, Not Active, Active",
        "0, 2032, 2032, 700.5, 0x0000000000000000, Not Active, Not Active, Not Active, Not Active",
    ]
    s = _sampler(lines)
    rec = s.stop()
    assert s.proc.terminated
    assert rec["sm_mhz"] == 2032.0 and rec["sm_max_mhz"] == 2032.0 and rec["samples"] == 3
    assert rec["reasons"] == ["sw_power_cap"]


def test_clock_record_every_rejecting_reason_is_seen():
    lines = [
        "0, 1500, 2032, 900.0, 0x08, Active, Not Active, Not Active, Not Active",
        "0, 1400, 2032, 900.0, 0x40, Not Active, Active, Not Active, Not Active",
        "0, 1600, 2032, 900.0, 0x20, Not Active, Not Active, Active, Not Active",
        "garbage line",
        "0, [N/A], 2032, 900.0, 0x0, Not Active, Not Active, Not Active, Not Active",
    ]
    rec = _sampler(lines).stop()
    assert rec["reasons"] == ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown"]
    assert rec["samples"] == 3 and rec["sm_mhz"] == 1500.0  # unparsable lines are skipped


def test_clock_record_without_a_sampler():
    s = bench.ClockSampler(0)  # start() never ran, as when nvidia-smi is missing
    rec = s.stop()
    assert rec["sm_mhz"] is None and rec["reasons"] == ["nvidia-smi unavailable"]


def test_oracle_samples_are_bounded_and_deterministic():
    for wl, n_ref, n_base in (("plain", 96, 1024), ("uneven", 256, 1024)):
        args = argparse.Namespace(workload=wl)
        sb1, desc1 = bench.oracle_sample(args)
        sb2, desc2 = bench.oracle_sample(args)
        assert desc1 == desc2 and np.array_equal(sb1.samples, sb2.samples)
        assert 0 < sb1.S <= n_ref
        if wl == "uneven":  # the oracle's O(T N) cost per segment stays bounded per series
            assert (sb1.steps.astype(np.float64) ** 2 * sb1.m < 2e8).all()
        base, _ = bench.oracle_sample(args, baseline=True)
        assert sb1.S <= base.S <= n_base


def test_workload_config_keys():
    for name in bench.WORKLOADS:
        c = bench.workload_config(name, 1, bench.WORKLOADS[name][2])
        assert {"workload", "series_per_gpu", "global_series", "l2", "parallelism"} <= set(c)
        assert "model" not in c
