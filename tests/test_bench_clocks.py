"""bench.py's clock record, with a stand-in for nvidia-smi on PATH (a shell
script that prints fixed samples): the first sample is dropped (it precedes
the timed region), the SM clock is the median of the rest, and every throttle
reason seen Active in any kept sample is reported."""
import os
import stat
import sys
import time
from pathlib import Path

ROOT = Path(__file__).resolve().parent.parent

SAMPLES = [
    # index, sm, max sm, power, active mask, hw, hw thermal, sw thermal, sw power cap
    "0, 900, 2070, 300.0, 0x0000000000000001, Not Active, Not Active, Not Active, Not Active",
    "0, 2070, 2070, 900.5, 0x0000000000000000, Not Active, Not Active, Not Active, Not Active",
    "0, 2040, 2070, 1390.0, 0x0000000000000004, Not Active, Not Active, Not Active, Active",
    "0, 2055, 2070, 1200.0, 0x0000000000000000, Not Active, Not Active, Not Active, Not Active",
]


def _fake_smi(tmp_path, lines):
    script = tmp_path / "nvidia-smi"
    body = "\n".join(f"echo '{line}'" for line in lines)
    script.write_text(f"#!/bin/sh\n{body}\nexec sleep 30\n")
    script.chmod(script.stat().st_mode | stat.S_IXUSR)
    return tmp_path


def _wait_for(cs, n_lines):
    # the stand-in writes all its samples at once; wait until they are on disk
    t0 = time.perf_counter()
    while time.perf_counter() - t0 < 10.0:
        if len(Path(cs.path).read_text().splitlines()) >= n_lines:
            return
        time.sleep(0.01)


def test_clock_record_from_samples(tmp_path, monkeypatch):
    sys.path.insert(0, str(ROOT))
    import bench
    monkeypatch.setenv("PATH", str(_fake_smi(tmp_path, SAMPLES)) + os.pathsep + os.environ["PATH"])
    cs = bench.ClockSampler(0)
    cs.start()
    assert cs.proc is not None
    _wait_for(cs, len(SAMPLES))
    rec = cs.stop()
    assert rec == {"sm_mhz": 2055.0, "sm_max_mhz": 2070.0, "reasons": ["sw_power_cap"],
                   "samples": 3}


def test_clock_record_reports_thermal_slowdown(tmp_path, monkeypatch):
    sys.path.insert(0, str(ROOT))
    import bench
    lines = SAMPLES[:2] + [
        "0, 1500, 2070, 1400.0, 0x0000000000000040, Not Active, Not Active, Active, Not Active"]
    monkeypatch.setenv("PATH", str(_fake_smi(tmp_path, lines)) + os.pathsep + os.environ["PATH"])
    cs = bench.ClockSampler(0)
    cs.start()
    _wait_for(cs, len(lines))
    rec = cs.stop()
    assert rec["reasons"] == ["sw_thermal_slowdown"]
    assert rec["sm_mhz"] == (2070.0 + 1500.0) / 2 and rec["samples"] == 2


def test_no_nvidia_smi_gives_no_record(tmp_path, monkeypatch):
    sys.path.insert(0, str(ROOT))
    import bench
    monkeypatch.setenv("PATH", str(tmp_path))
    cs = bench.ClockSampler(0)
    cs.start()
    assert cs.stop() is None
