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


def _json_lines(out):
    import json

    return [json.loads(l) for l in out.splitlines() if l.startswith("{")]


def test_reference_arm_prints_one_line():
    """bench.py --impl reference: the oracle as the reference arm, one JSON line
    with the contract's keys (runs on host cores only)."""
    import subprocess
    import sys

    r = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--steps", "1", "--warmup", "1"],
                       cwd=ROOT, capture_output=True, text=True, timeout=900)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = _json_lines(r.stdout)
    assert len(lines) == 1
    d = lines[0]
    for k in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better", "config",
              "cpu_baseline", "e2e"):
        assert k in d, k
    assert d["impl"] == "reference" and d["unit"] == "checks/s" and d["value"] > 0
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["cores"] >= 1
    assert d["e2e"]["h2d_bytes_per_step"] == 0 and d["e2e"]["d2h_bytes_per_step"] == 0


def test_reference_arm_under_torchrun_two_ranks():
    """Launched as the multi-GPU bench is (torchrun, 127.0.0.1): rank 0 alone
    runs the oracle and prints; the other rank exits 0 without work."""
    import socket
    import subprocess
    import sys

    with socket.socket() as so:
        so.bind(("127.0.0.1", 0))
        port = so.getsockname()[1]
    r = subprocess.run([sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node", "2",
                        "--master-addr", "127.0.0.1", "--master-port", str(port), "bench.py", "--impl", "reference",
                        "--gpus", "2", "--steps", "1", "--warmup", "1"],
                       cwd=ROOT, capture_output=True, text=True, timeout=900)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = _json_lines(r.stdout)
    assert len(lines) == 1 and lines[0]["impl"] == "reference"
