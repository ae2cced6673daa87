"""Host logic of bench.py that needs no GPU: the clock sampler against a stand-in
nvidia-smi (a script on PATH printing the queried CSV fields), so the parsing of
clocks and throttle reasons, and the wait for the first sample, run on CPU."""
from __future__ import annotations

import importlib.util
import os
import stat
import time

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def load_bench():
    spec = importlib.util.spec_from_file_location("bench_under_test", os.path.join(ROOT, "bench.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


FAKE = """#!/bin/sh
# stand-in for nvidia-smi -lms: a short start-up, then one CSV line per tick
sleep 0.3
i=0
while [ $i -lt 200 ]; do
  echo "0, {mhz}, 2070, 900.5, 0x0, Not Active, Not Active, Not Active, {cap}"
  i=$((i + 1))
  sleep 0.02
done
"""


@pytest.mark.parametrize("mhz,cap,reasons", [(2070, "Not Active", []), (1980, "Active", ["sw_power_cap"])])
def test_clock_sampler_parses_a_fake_nvidia_smi(tmp_path, monkeypatch, mhz, cap, reasons):
    exe = tmp_path / "nvidia-smi"
    exe.write_text(FAKE.format(mhz=mhz, cap=cap))
    exe.chmod(exe.stat().st_mode | stat.S_IXUSR)
    monkeypatch.setenv("PATH", f"{tmp_path}{os.pathsep}{os.environ['PATH']}")
    bench = load_bench()
    s = bench.ClockSampler(0)
    t0 = time.time()
    s.start()
    waited = time.time() - t0
    assert 0.25 <= waited < 3.0  # returned after the first sample, not before
    time.sleep(0.2)
    r = s.stop()
    assert r["sm_mhz"] == mhz and r["sm_max_mhz"] == 2070 and r["reasons"] == reasons and r["samples"] >= 2


def test_clock_sampler_without_nvidia_smi(tmp_path, monkeypatch):
    monkeypatch.setenv("PATH", str(tmp_path))  # nothing to run
    bench = load_bench()
    s = bench.ClockSampler(0)
    s.start()
    assert s.stop() is None
