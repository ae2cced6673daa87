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


def test_roofline_fraction_is_bounded_and_reproducible():
    """The bench line's roofline.frac comes from the work the kernel executed
    on the unit that bounds it: for the profiled launch itself (its evaluated
    checks over its own duration) it reproduces the busy fraction the profile
    measured (shared-memory wavefronts for the nibble-table search, the ALU
    pipe for the bit-plane search) and it is below 1; the (N-K)/32-ops-per-check
    model figure is kept apart (model_ops)."""
    bench = load_bench()
    cfg = dict(bench.CONFIGS["c2"], name="c2")
    assert bench.search_kernel(cfg) == ("k_search_warp", "k_search_warp S'<=10")
    prof = bench.NCU_SEARCH["k_search_warp S'<=10"]
    # the profiled small case: 1.00e10 evaluated checks in 143.1 us at 2.07 GHz
    r = bench.search_roofline(cfg, 10032515195.0, 8800799405.0, 11181, 0.143072, 2.0)
    assert r["kernel"] == "k_search_warp" and r["bound"] == "smem" and r["unit"] == "GB/s"
    assert 0.5 < r["frac"] < 1.0
    assert abs(r["frac"] - prof["smem_wavefronts_frac"]) < 0.02
    assert 0.0 < r["alu"]["frac"] < 1.0
    assert r["model_ops"]["frac"] > 1.0  # the per-useful-check cost model is not a fraction of a pipe
    cfg3 = dict(bench.CONFIGS["c3a"], name="c3a")
    assert bench.search_kernel(cfg3) == ("k_search_warp", "k_search_warp S'=12")
    r3 = bench.search_roofline(cfg3, 78007607510.0, 77714307970.0, 4706, 0.901472, 8.0)
    assert r3["bound"] == "smem"
    assert abs(r3["frac"] - bench.NCU_SEARCH["k_search_warp S'=12"]["smem_wavefronts_frac"]) < 0.02
    cfg1 = dict(bench.CONFIGS["c1"], name="c1")
    assert bench.search_kernel(cfg1)[0] == "k_ab_split<1,16>"


def test_adversarial_mix_keeps_the_batch_consistent():
    """The serving mix with a hard share: the offsets stay consistent, the
    chosen frames are N=1024 at 4 dB, the other frames' symbols and codewords
    are the original mix's."""
    import numpy as np

    import oracle
    import workloads as wl

    bench = load_bench()
    info = {n: oracle.info_set(n, n // 2) for n in wl.MIXED_N}
    mx = wl.mixed_frames(8, 1000, 4000, info)
    a = bench.with_hard_share(mx, 8, 0, 0.25, info)
    F = 4000
    assert int(a["hard"].sum()) == 1000
    assert np.all(a["N"][a["hard"]] == 1024) and np.all(a["ebn0_db"][a["hard"]] == 4.0)
    L = np.array([wl.symbols_per_frame(int(n), int(m)) for n, m in zip(a["N"], a["M"])])
    assert np.array_equal(a["L"], L)
    assert np.array_equal(np.diff(np.append(a["sym_offset"], a["n_sym"])), L)
    assert np.array_equal(np.diff(np.append(a["cw_offset"], a["n_cw_words"])), a["N"] // 32)
    for f in np.nonzero(~a["hard"])[0][:200]:
        so, mo, n = a["sym_offset"][f], mx["sym_offset"][f], L[f]
        assert np.array_equal(a["symbols"][so:so + n], mx["symbols"][mo:mo + n])
        co, mc, w = a["cw_offset"][f], mx["cw_offset"][f], a["N"][f] // 32
        assert np.array_equal(a["codewords_packed"][co:co + w], mx["codewords_packed"][mc:mc + w])
    # a hard frame's symbols are a valid 1024-bit codeword's transmission (decodable at high SNR is
    # not the point here: its codeword satisfies H c = 0)
    H = oracle.parity_H(1024, 512)
    f = np.nonzero(a["hard"])[0][0]
    c = a["codewords_packed"][a["cw_offset"][f]:a["cw_offset"][f] + 32]
    bits = ((c[:, None] >> np.arange(32, dtype=np.uint32)) & 1).reshape(-1).astype(np.int64)
    assert not ((H.astype(np.int64) @ bits) % 2).any()
