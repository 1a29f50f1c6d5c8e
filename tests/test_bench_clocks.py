"""bench.py's clock sampler, on CPU, against a stand-in nvidia-smi.

The stand-in prints rows in nvidia-smi's query format (timestamp first) at
the requested period, optionally with hw_slowdown active, and buffers its
output like a program writing to a pipe does, so the sampler has to rely on
the timestamps, not on when the rows arrive."""
import os
import stat
import sys
import time

import bench

FAKE = r'''#!{python}
import datetime, os, sys, time
period = 0.05
args = sys.argv[1:]
if "-lms" in args:
    period = int(args[args.index("-lms") + 1]) / 1000.0
slow = os.environ.get("FAKE_SMI_SLOWDOWN") == "1"
out = sys.stdout
while True:
    ts = datetime.datetime.now().strftime("%Y/%m/%d %H:%M:%S.%f")[:-3]
    hw = "Active" if slow else "Not Active"
    out.write(f"{{ts}}, 0, 1965, 2070, 812.50, 0x0000000000000000, {{hw}}, Not Active, Not Active, Not Active\n")
    time.sleep(period)
'''


def _install(tmp_path, monkeypatch, slowdown=False):
    path = tmp_path / "nvidia-smi"
    path.write_text(FAKE.format(python=sys.executable))
    path.chmod(path.stat().st_mode | stat.S_IEXEC)
    monkeypatch.setenv("PATH", f"{tmp_path}{os.pathsep}{os.environ['PATH']}")
    monkeypatch.setenv("FAKE_SMI_SLOWDOWN", "1" if slowdown else "0")


def test_rows_inside_the_region_only(tmp_path, monkeypatch):
    _install(tmp_path, monkeypatch)
    with bench.ClockSampler(0) as c:
        time.sleep(0.5)
    s = c.summary()
    # about 500 / PERIOD_MS rows; the bound leaves room for a slow host
    n = 500 / bench.ClockSampler.PERIOD_MS
    assert 0.4 * n <= s["samples"] <= 1.3 * n
    assert s["sm_mhz"] == 1965.0 and s["sm_max_mhz"] == 2070.0
    assert s["reasons"] == [] and "note" not in s
    assert 450 <= s["window_ms"] <= 2000


def test_slowdown_reason_reported(tmp_path, monkeypatch):
    _install(tmp_path, monkeypatch, slowdown=True)
    with bench.ClockSampler(0) as c:
        time.sleep(0.2)
    assert c.summary()["reasons"] == ["hw_slowdown"]


def test_region_shorter_than_the_period_keeps_the_nearest_row(tmp_path, monkeypatch):
    _install(tmp_path, monkeypatch)
    monkeypatch.setattr(bench.ClockSampler, "PERIOD_MS", 400)
    with bench.ClockSampler(0) as c:
        pass
    s = c.summary()
    assert s["samples"] == 1 and "note" in s and s["sm_mhz"] == 1965.0


def test_missing_nvidia_smi(tmp_path, monkeypatch):
    monkeypatch.setenv("PATH", str(tmp_path))
    with bench.ClockSampler(0) as c:
        pass
    s = c.summary()
    assert s["samples"] == 0 and s["sm_mhz"] is None
