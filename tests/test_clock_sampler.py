"""bench.py's clock record (no GPU needed): a stand-in nvidia-smi on PATH prints
samples in the CSV layout of the query every -lms milliseconds; the sampler keeps
those stamped inside the timed region (a region of 100 ms still holds several),
reports throttle reasons, and gives an empty record when the tool is missing."""
import os
import sys
import time

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

FAKE = r"""#!/usr/bin/env python3
import datetime, os, signal, sys, time
args = sys.argv[1:]
lms = int(args[args.index("-lms") + 1]) if "-lms" in args else 1000
hw = "Active" if os.environ.get("FAKE_SMI_MODE") == "hw" else "Not Active"
stop = []
signal.signal(signal.SIGINT, lambda *a: stop.append(1))
while not stop:
    ts = datetime.datetime.now().strftime("%Y/%m/%d %H:%M:%S.%f")[:-3]
    print(f"{ts}, 2070, 2070, 812.50, 0x0000000000000000, {hw}, Not Active, Not Active, Not Active",
          flush=True)
    time.sleep(lms / 1000.0)
"""


@pytest.fixture()
def bench_mod():
    sys.path.insert(0, ROOT)
    import bench
    return bench


def _fake_tool(tmp_path, monkeypatch, mode):
    d = tmp_path / "bin"
    d.mkdir()
    f = d / "nvidia-smi"
    f.write_text(FAKE)
    f.chmod(0o755)
    monkeypatch.setenv("PATH", str(d) + os.pathsep + os.environ.get("PATH", ""))
    monkeypatch.setenv("FAKE_SMI_MODE", mode)


def test_short_region_holds_samples(bench_mod, tmp_path, monkeypatch):
    _fake_tool(tmp_path, monkeypatch, "ok")
    with bench_mod.ClockSampler(0) as clk:
        time.sleep(0.1)
    s = clk.summary()
    assert s["window"] == "timed region"
    assert 2 <= s["samples"] <= 10
    assert s["sm_mhz"] == 2070.0 and s["sm_max_mhz"] == 2070.0 and s["reasons"] == []
    # samples taken before the region (the sampler's start-up) are not counted
    assert len(clk.lines) >= s["samples"]


def test_throttle_reason_is_reported(bench_mod, tmp_path, monkeypatch):
    _fake_tool(tmp_path, monkeypatch, "hw")
    with bench_mod.ClockSampler(0) as clk:
        time.sleep(0.06)
    assert "hw_slowdown" in clk.summary()["reasons"]


def test_without_the_tool(bench_mod, tmp_path, monkeypatch):
    monkeypatch.setenv("PATH", str(tmp_path))
    with bench_mod.ClockSampler(0) as clk:
        pass
    s = clk.summary()
    assert s["samples"] == 0 and s["sm_mhz"] is None and s["reasons"] == []
