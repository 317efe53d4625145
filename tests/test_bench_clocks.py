"""bench.py's clock record (median SM clock under load, maximum clock and the
throttle reasons seen during the timed region), checked against a stand-in
`nvidia-smi` that prints fixed samples; and the record when the tool is
missing."""

import os
import stat
import time

import bench

SAMPLES = [
    "0, 2070, 2070, 650.1, 0x0000000000000000, Not Active, Not Active, Not Active, Not Active",
    "0, 1980, 2070, 1390.0, 0x0000000000000004, Not Active, Not Active, Not Active, Active",
    "0, 2055, 2070, 900.0, 0x0000000000000000, Not Active, Not Active, Not Active, Not Active",
    "garbage line",
    "0, [N/A], 2070, 900.0, 0x0, Not Active, Not Active, Not Active, Not Active",
]


def _fake_smi(tmp_path, lines):
    exe = tmp_path / "nvidia-smi"
    body = "".join(f"printf '%s\\n' '{line}'\n" for line in lines)
    exe.write_text("#!/bin/bash\n" + body + "exec sleep 30\n")
    exe.chmod(exe.stat().st_mode | stat.S_IXUSR)
    return str(tmp_path)


def test_clock_record_from_samples(tmp_path, monkeypatch):
    monkeypatch.setenv("PATH", _fake_smi(tmp_path, SAMPLES) + os.pathsep + os.environ["PATH"])
    s = bench.ClockSampler(0)
    s.start()
    time.sleep(0.5)
    rec = s.stop()
    assert rec["samples"] == 3
    assert rec["sm_mhz"] == 2055.0 and rec["sm_max_mhz"] == 2070.0
    assert rec["reasons"] == ["sw_power_cap"]


def test_clock_record_reports_each_slowdown(tmp_path, monkeypatch):
    lines = ["0, 1500, 2070, 1400.0, 0x0, Active, Not Active, Active, Not Active"]
    monkeypatch.setenv("PATH", _fake_smi(tmp_path, lines) + os.pathsep + os.environ["PATH"])
    s = bench.ClockSampler(0)
    s.start()
    time.sleep(0.5)
    rec = s.stop()
    assert rec["reasons"] == ["hw_slowdown", "sw_thermal_slowdown"] and rec["sm_mhz"] == 1500.0


def test_clock_record_without_the_tool(tmp_path, monkeypatch):
    monkeypatch.setenv("PATH", str(tmp_path))
    s = bench.ClockSampler(0)
    s.start()
    rec = s.stop()
    assert rec["sm_mhz"] is None and rec["reasons"] in (["nvidia-smi unavailable"], ["no samples"])
