"""Host-side pieces of bench.py that need no GPU: the clock record that goes beside
every timed number (median SM clock, throttle reasons) and its sample file."""
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402


def test_clock_summary_reads_reasons_and_removes_its_samples():
    c = bench.ClockSampler(0)
    c.proc = object()  # as if nvidia-smi had run: parse the file it would have written
    with open(c.path, "w") as f:
        f.write("0, 2070, 2070, 400.5, 0x0, Not Active, Not Active, Not Active, Active\n")
        f.write("0, 1980, 2070, 410.0, 0x0, Not Active, Not Active, Not Active, Not Active\n")
        f.write("0, 2070, 2070, 420.0, 0x0, Active, Not Active, Not Active, Not Active\n")
        f.write("garbage line\n")
    s = c.summary()
    assert s["sm_mhz"] == 2070.0 and s["sm_max_mhz"] == 2070.0 and s["samples"] == 3
    assert s["power_w_median"] == 410.0
    assert s["reasons"] == ["hw_slowdown", "sw_power_cap"]
    assert not os.path.exists(c.path)
    assert c.summary() == s  # read once


def test_clock_sampler_without_nvidia_smi_leaves_no_file(monkeypatch):
    def missing(*a, **k):
        raise FileNotFoundError("nvidia-smi")

    monkeypatch.setattr(bench.subprocess, "Popen", missing)
    c = bench.ClockSampler(0)
    with c:
        pass
    assert c.summary()["reasons"] == ["nvidia-smi unavailable"]
    assert not os.path.exists(c.path)

