"""Host-side pieces of the benchmark that need no GPU: the clock sampler's
parsing of nvidia-smi lines and its subprocess plumbing (with a stand-in
nvidia-smi on PATH that prints fixed lines)."""
from __future__ import annotations

import os
import stat
import time


def test_clock_summary_parses_samples_and_reasons():
    import bench

    s = bench.ClockSampler(0)
    s.lines = [
        "0, 2070, 2070, 910.25, 0x0000000000000000, Not Active, Not Active, Not Active, Not Active",
        "0, 1995, 2070, 1390.00, 0x0000000000000004, Not Active, Not Active, Not Active, Active",
        "0, 2070, 2070, 1200.10, 0x0000000000000000, Not Active, Not Active, Not Active, Not Active",
        "0, [N/A], 2070, 10.0, 0x0, Not Active, Not Active, Not Active, Not Active",  # skipped
        "garbage",
    ]
    got = s.summary()
    assert got == {"sm_mhz": 2070.0, "sm_max_mhz": 2070.0, "reasons": ["sw_power_cap"], "samples": 3}
    s.lines = ["0, 1200, 2070, 500, 0x8, Active, Not Active, Active, Not Active"]
    assert s.summary()["reasons"] == ["hw_slowdown", "sw_thermal_slowdown"]
    s.lines = []
    assert s.summary() is None


def test_clock_sampler_reads_a_running_tool(tmp_path, monkeypatch):
    import bench

    fake = tmp_path / "nvidia-smi"
    fake.write_text("#!/bin/sh\n"
                    "echo '0, 2070, 2070, 900, 0x0, Not Active, Not Active, Not Active, Not Active'\n"
                    "echo '0, 2055, 2070, 950, 0x0, Not Active, Not Active, Not Active, Not Active'\n"
                    "exec sleep 30\n")
    fake.chmod(fake.stat().st_mode | stat.S_IXUSR)
    monkeypatch.setenv("PATH", f"{tmp_path}{os.pathsep}{os.environ['PATH']}")
    with bench.ClockSampler(0) as s:
        t0 = time.time()
        while len(s.lines) < 2 and time.time() - t0 < 10:
            time.sleep(0.05)
    got = s.summary()
    assert got["samples"] == 2 and got["sm_max_mhz"] == 2070.0 and got["reasons"] == []
    assert s.proc.poll() is not None  # the sampler stopped its tool


def test_clock_sampler_without_the_tool(tmp_path, monkeypatch):
    import bench

    monkeypatch.setenv("PATH", str(tmp_path))
    with bench.ClockSampler(0) as s:
        pass
    assert s.summary() is None
