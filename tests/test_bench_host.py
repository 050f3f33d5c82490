"""Host logic of bench.py on the CPU: the clock sampler's record (median SM clock, the maximum,
the throttle reasons seen active) from a stand-in for the sampling tool that prints the same
CSV rows, and its bounded wait for the first sample before the timed region."""
import os
import stat
import sys
import time

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
import bench  # noqa: E402

ROWS = [
    "0, 2070, 2070, 900.1, 0x0, Not Active, Not Active, Not Active, Not Active",
    "0, 1980, 2070, 1390.5, 0x4, Not Active, Not Active, Not Active, Active",
    "0, 2070, 2070, 1200.0, 0x0, Not Active, Not Active, Not Active, Not Active",
]


def _fake_tool(tmp_path, rows, delay_s):
    exe = tmp_path / "fake-smi"
    body = "\n".join(f"    print({r!r}, flush=True)\n    time.sleep(0.05)" for r in rows) or "    pass"
    exe.write_text(f"#!{sys.executable}\nimport time\ntime.sleep({delay_s})\nif True:\n{body}\n")
    exe.chmod(exe.stat().st_mode | stat.S_IEXEC)
    return str(exe)


def test_clock_record_from_rows(tmp_path):
    exe = _fake_tool(tmp_path, ROWS, 0.3)
    with bench.ClockSampler(0, exe=exe) as clk:
        assert clk.lines, "the first sample should have arrived before the timed region"
        time.sleep(0.5)
    s = clk.summary()
    assert s["samples"] == 3
    assert s["sm_mhz"] == 2070.0 and s["sm_max_mhz"] == 2070.0
    assert s["reasons"] == ["sw_power_cap"]


def test_missing_tool_and_silent_tool(tmp_path):
    with bench.ClockSampler(0, exe=str(tmp_path / "absent")) as clk:
        pass
    assert clk.summary() == {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
    exe = _fake_tool(tmp_path, [], 5.0)          # prints nothing: the wait is bounded
    t = time.perf_counter()
    with bench.ClockSampler(0, exe=exe, first_wait_s=0.3) as clk:
        pass
    assert time.perf_counter() - t < 3.0
    assert clk.summary()["samples"] == 0
