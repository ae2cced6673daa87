#!/usr/bin/env python3
"""Benchmark of the GB300 GRAND decoder (arXiv 2405.01808, Alg. 2 on a GPU).

Default workload: polar code N=128 K=64 (Bhattacharyya frozen set at 0 dB), Gray
16-QAM over AWGN at Eb/N0 = 6, 8 and 10 dB, 100,000 frames per SNR (300,000
frames per step), cut-off S = 10, query cap 2^20, symbol-level TEP order of the
paper's likelihood function. One step decodes the whole batch through the
fused demodulate-and-decode call (grand_decode_symbols): demodulation,
likelihood and neighbours, selection, syndrome deltas, TEP enumeration and
membership tests, and the decoded words.

Metric: useful TEP syndrome checks per second (the sum of the query counts,
i.e. valid TEPs up to the first codeword or the cap), with frames/s and the
per-step latency beside it. Inputs are resident in HBM; L2 is flushed (256 MiB
write) before every timed step. `e2e` repeats the measurement through the same
public call with pinned host buffers (copies in the timed region).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]
                  [--config c1|c2|c3a|c3b|c4]
"""
from __future__ import annotations

import argparse
import gc
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import workloads as wl  # noqa: E402

# -------------------------------------------------------------------------
# workloads
# -------------------------------------------------------------------------
CONFIGS = {
    "c1": dict(kind="ab", N=32, K=16, M=2, snrs=(4.0,), frames=10000, max_weight=3, cap=5489,
               desc="polar N=32 K=16, BPSK, Eb/N0 4 dB, GRAND-AB weight<=3 (cap 5489), 10000 frames"),
    "c2": dict(kind="qam", N=128, K=64, M=16, snrs=(6.0, 8.0, 10.0), frames=100000, S=10, cap=1 << 20,
               desc="polar N=128 K=64, 16-QAM Gray, Eb/N0 6/8/10 dB x 100000 frames, S=10, cap 2^20"),
    "c3a": dict(kind="qam", N=512, K=256, M=64, snrs=(10.0, 12.0, 14.0, 16.0), frames=20000, S=12, cap=1 << 24,
                desc="polar N=512 K=256, 64-QAM Gray, Eb/N0 10/12/14/16 dB x 20000 frames, S=12, cap 2^24"),
    "c3b": dict(kind="qam", N=1024, K=512, M=256, snrs=(10.0, 12.0, 14.0, 16.0), frames=20000, S=12, cap=1 << 24,
                desc="polar N=1024 K=512, 256-QAM Gray, Eb/N0 10/12/14/16 dB x 20000 frames, S=12, cap 2^24"),
    "c4": dict(kind="mixed", frames=1000000, S=10, cap=1 << 20,
               desc="uneven mix: N in {32..1024}, M in {4,16,64,256}, Eb/N0 U(4,14) dB, 1000000 frames, "
                    "S=min(L,10), cap 2^20, one call"),
    "bler": dict(kind="bler", frames=1000000, S=8,
                 desc="BLER vs Eb/N0 at S=8 (the paper's cut-off), cap 4^8: N in {32..1024} x M in {4..4096}, "
                      "Eb/N0 grid of 9 points per M, frames per point as given"),
    "orders": dict(kind="orders", N=128, K=64, M=16, snrs=(6.0, 8.0, 10.0), frames=20000,
                   desc="TEP order comparison on polar N=128 K=64, 16-QAM, Eb/N0 6/8/10 dB x 20000 frames: the "
                        "paper's order, its literal Def. III.1 reading, nearer axis first, five-point NNE; S=8 "
                        "with the whole space (4^8 / 5^8) and S=10 with cap 2^20"),
    "membership": dict(kind="membership", N=128, K=64, M=16, snrs=(6.0, 8.0, 10.0), frames=2000, S=10,
                       cap=1 << 20,
                       desc="membership-test ablation on polar N=128 K=64, 16-QAM, Eb/N0 6/8/10 dB x 2000 "
                            "frames, S=10, cap 2^20: split search (syndrome deltas, bit-sliced), per-TEP "
                            "syndrome deltas, per-TEP row parity (Alg. 1's product)"),
    "c5": dict(kind="serve", frames=1000000, S=10, cap=1 << 20, rates=(0.5e6, 1e6, 2e6, 5e6),
               desc="serving: Poisson arrivals at 0.5/1/2/5 M frames/s of the uneven mix (N 32..1024, "
                    "M 4..256, Eb/N0 U(4,14) dB), 1000000 requests per rate, S=min(L,10), cap 2^20"),
    "c5long": dict(kind="serve", frames=200000, S=12, cap=1 << 24, rates=(0.5e6,), adversarial=0.02,
                   ebn0=(8.0, 14.0),
                   desc="serving, long frames: the uneven mix at Eb/N0 U(8,14) dB with 2 % of the requests "
                        "replaced by N=1024 frames at 4 dB, S=min(L,12), cap 2^24 (a long frame searches up to "
                        "16.8 M TEPs), Poisson 0.5 M frames/s, 200000 requests; long frames whole in their batch "
                        "vs continued from device-resident cursors after their batch is reported"),
    "c5adv": dict(kind="serve", frames=400000, S=10, cap=1 << 20, rates=(1e6,), adversarial=0.25,
                  desc="serving, adversarial mix: the uneven mix with a quarter of the requests replaced by "
                       "N=1024 frames at Eb/N0 4 dB (most search their whole 2^20 queries), Poisson 1 M frames/s, "
                       "400000 requests; long frames whole in their batch vs carried as device-resident cursors"),
}
METRIC = "TEP syndrome checks/s & frames/s per GB300; p50/p99 decode latency"
CONFIG_IDS = {"c1": 1, "c2": 2, "c3a": 3, "c3b": 4, "c4": 5, "c5": 6, "c5adv": 8, "c5long": 9, "bler": 7, "orders": 2,
              "membership": 2}
# ALU roofline: 152 SMs x 64 integer-ALU lanes per clock (LOP3/ISETP class)
# x 2.07 GHz maximum SM clock.
SMS, ALU_LANES, MAX_CLOCK_GHZ = 152, 64, 2.07
ALU_PEAK_TOPS = SMS * ALU_LANES * MAX_CLOCK_GHZ / 1000.0
# Shared-memory roofline: one 128-byte wavefront per clock per SM (32 banks x
# 4 B; ncu's l1tex data-pipe peak), 152 SMs x 2.07 GHz.
SMEM_PEAK_GBS = SMS * 128 * MAX_CLOCK_GHZ
# Counters of each search kernel from one ncu capture of a small case (the
# profiles/ file named), taken on the decode.cu source with the given sha256
# prefix. Per TEP check the kernel evaluated in that launch:
#   smem_bytes_per_check = shared-memory wavefronts x 128 B / checks (the
#     warp search reads three table words per 32 TEPs per lane: it is bound
#     by shared-memory bandwidth);
#   alu_lane_ops_per_check = ALU pipe busy fraction x elapsed cycles x SMs x
#     64 lanes / checks (the bit-level GRAND-AB kernel is bound by the integer
#     pipe).
# Everything in the kernel is included in both.
NCU_SEARCH = {
    "k_search_warp S'<=10": {"sha": "c0a370e5b6a95e2b", "profile": "profiles/k_search_warp_c2_small.md",
                             "bound": "smem", "smem_bytes_per_check": 0.4489, "smem_wavefronts_frac": 0.778,
                             "lsu_pipe_active": 0.820, "alu_lane_ops_per_check": 0.147, "alu_pipe_active": 0.511,
                             "dram_bytes_per_hard_frame": 1894912 / 11181},
    "k_search_warp S'=12": {"sha": "c0a370e5b6a95e2b", "profile": "profiles/k_search_warp_c3a_small.md",
                            "bound": "smem", "smem_bytes_per_check": 0.4059, "smem_wavefronts_frac": 0.867,
                            "lsu_pipe_active": 0.904, "alu_lane_ops_per_check": 0.104, "alu_pipe_active": 0.443,
                            "dram_bytes_per_hard_frame": 777216 / 4706},
    # the bit-level kernel reads every frame (no hand-off records): bytes per frame
    "k_ab_split<1,16>": {"sha": "c0a370e5b6a95e2b", "profile": "profiles/k_ab_split_c1_n32_bpsk.md", "bound": "alu",
                         "alu_lane_ops_per_check": 162.4, "alu_pipe_active": 0.349,
                         "dram_bytes_per_frame": 1308416 / 10000},
}


def decode_source_sha():
    import hashlib

    with open(os.path.join(ROOT, "paper_2405_01808_gb300", "csrc", "decode.cu"), "rb") as fh:
        return hashlib.sha256(fh.read()).hexdigest()[:16]


def search_kernel(cfg):
    """The kernel that runs the TEP search of a workload with automatic tiles,
    and the key of its profile (the flip-bit search is profiled at S' <= 10
    and at S' = 12, whose B side is 16 times larger)."""
    if cfg["kind"] == "ab":
        k = "k_ab_split<1,16>" if cfg["N"] == 32 else "k_ab"
        return k, k
    return "k_search_warp", ("k_search_warp S'=12" if cfg["S"] > 10 else "k_search_warp S'<=10")


def search_roofline(cfg, evaluated, useful, hard, kernel_ms, alg_words, frames=0):
    """Roofline of the TEP search kernel against the peak of the unit that
    bounds it: shared-memory bandwidth for the nibble-table search (S' <= 10),
    the integer ALU for the bit-plane searches (S' = 11, 12; GRAND-AB).

    frac = the kernel's use of that unit per second / its peak, with the use =
    TEP checks the kernel evaluated in this run (counted on the device) x what
    one evaluated check costs the unit (ncu, same kernel: shared-memory bytes
    or ALU lane-ops). It stays below 1 by construction. The per-check cost
    model of (N-K)/32 three-input ops per useful check is kept beside it as model_ops:
    it can exceed the ALU peak, because the split compare tests 32 TEPs per
    table word or logic op on a projection and confirms only matches on the
    full syndrome."""
    kern, prof_key = search_kernel(cfg)
    prof = NCU_SEARCH.get(prof_key)
    t_s = kernel_ms / 1e3
    alu_src = (f"derived: {SMS} SMs x {ALU_LANES} ALU lanes/clk x {MAX_CLOCK_GHZ} GHz (a LOP3 microbenchmark on "
               "this GPU measured 64 per clock per SM)")
    smem_src = f"derived: {SMS} SMs x 128 B/clk (one shared-memory wavefront) x {MAX_CLOCK_GHZ} GHz"
    bound = prof.get("bound", "alu") if prof else "alu"
    rec = {"bound": bound, "kernel": kern, "kernel_ms": kernel_ms, "evaluated_checks": evaluated,
           "useful_checks": useful}
    if bound == "smem":
        rec.update({"peak": SMEM_PEAK_GBS, "unit": "GB/s", "peak_source": smem_src})
    else:
        rec.update({"peak": ALU_PEAK_TOPS, "unit": "Tops/s", "peak_source": alu_src})
    if prof is not None:
        same = decode_source_sha() == prof["sha"]
        if "dram_bytes_per_frame" in prof:
            traffic = prof["dram_bytes_per_frame"] * frames if same and frames else None
        else:
            traffic = prof["dram_bytes_per_hard_frame"] * hard if same and hard else None
        alu_ach = evaluated * prof["alu_lane_ops_per_check"] / t_s / 1e12
        if bound == "smem":
            ach = evaluated * prof["smem_bytes_per_check"] / t_s / 1e9
            rec.update({"achieved": ach, "frac": ach / SMEM_PEAK_GBS,
                        "smem_bytes_per_evaluated_check": prof["smem_bytes_per_check"],
                        "derivation": "evaluated checks of this run x shared-memory bytes per evaluated check "
                                      "(ncu wavefronts x 128 B) / event-timed kernel time / shared-memory peak",
                        "ncu_smem_wavefronts_frac": prof["smem_wavefronts_frac"],
                        "ncu_lsu_pipe_active": prof["lsu_pipe_active"],
                        "alu": {"achieved": alu_ach, "peak": ALU_PEAK_TOPS, "unit": "Tops/s",
                                "frac": alu_ach / ALU_PEAK_TOPS,
                                "alu_lane_ops_per_evaluated_check": prof["alu_lane_ops_per_check"]}})
        else:
            rec.update({"achieved": alu_ach, "frac": alu_ach / ALU_PEAK_TOPS,
                        "alu_lane_ops_per_evaluated_check": prof["alu_lane_ops_per_check"],
                        "derivation": "evaluated checks of this run x ALU lane-ops per evaluated check (ncu) / "
                                      "event-timed kernel time / ALU peak"})
        rec.update({"traffic": traffic, "profile": prof["profile"], "profile_source_sha": prof["sha"],
                    "profile_matches_source": same, "ncu_alu_pipe_active": prof["alu_pipe_active"]})
    else:
        rec.update({"achieved": None, "frac": None, "traffic": None})
    if alg_words is not None:
        m = useful * alg_words / t_s / 1e12
        rec["model_ops"] = {"ops_per_useful_check": alg_words, "achieved": m, "frac": m / ALU_PEAK_TOPS,
                            "note": "(N-K)/32 three-input ops per useful check against the ALU peak; can exceed 1 "
                                    "(the split compare tests 32 TEPs per table word or logic op on a projection)"}
    return rec


def gpu_busy_us(us):
    """Keep the current stream busy for about `us` microseconds (a spin kernel),
    so that a kernel-level measurement whose events are recorded next does not
    include the host's time to issue the call (the GPU would sit idle between
    the first event and the launch)."""
    import torch

    try:
        torch.cuda._sleep(int(us * MAX_CLOCK_GHZ * 1000))
    except (AttributeError, RuntimeError):
        pass


def hbm_peak():
    """Measured copy bandwidth of this machine's GPUs (GB/s) and where it came from."""
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as fh:
            return float(json.load(fh)["hbm_gbs"]), "measured (MEASURED_PEAKS.json hbm_gbs)"
    except (OSError, KeyError, ValueError):
        return 6800.0, "fallback (6.8 TB/s)"


def make_inputs(cfg, rank, info_by_N):
    """Host arrays of one step's batch (seeded; rank selects the stream)."""
    from paper_2405_01808_gb300.dist import shard_stream

    if cfg["kind"] in ("bler", "orders", "membership"):
        return None
    cid = CONFIG_IDS[cfg["name"]]
    if cfg["kind"] in ("mixed", "serve"):
        mx = wl.mixed_frames(cid, 1000 + rank, cfg["frames"], info_by_N, ebn0_range=cfg.get("ebn0", (4.0, 14.0)))
        if cfg.get("adversarial"):
            mx = with_hard_share(mx, cid, rank, cfg["adversarial"], info_by_N)
        return mx
    parts = []
    for i, snr in enumerate(cfg["snrs"]):
        if cfg["kind"] == "ab":
            parts.append(wl.bpsk_frames(cid, shard_stream(rank, i), cfg["frames"], cfg["N"], info_by_N[cfg["N"]], snr))
        else:
            parts.append(wl.qam_frames(cid, shard_stream(rank, i), cfg["frames"], cfg["N"], info_by_N[cfg["N"]],
                                       cfg["M"], snr))
    return {"symbols": np.concatenate([p["symbols"] for p in parts]),
            "codewords_packed": np.concatenate([p["codewords_packed"] for p in parts]),
            "snr": np.concatenate([np.full(len(p["symbols"]), p["ebn0_db"]) for p in parts])}


def with_hard_share(mx, cid, rank, share, info_by_N):
    """Replace a share of the frames of an uneven batch (seeded positions) by
    N=1024 frames at Eb/N0 4 dB over the same constellation mix."""
    F = len(mx["N"])
    g = wl.rng(cid, 5000 + rank)
    hard = np.sort(g.choice(F, size=int(F * share), replace=False))
    hx = wl.mixed_frames(cid, 6000 + rank, len(hard), info_by_N, ebn0_range=(4.0, 4.0), n_choices=(1024,))
    N, M, snr = mx["N"].copy(), mx["M"].copy(), mx["ebn0_db"].copy()
    N[hard], M[hard], snr[hard] = hx["N"], hx["M"], hx["ebn0_db"]
    L = np.array([wl.symbols_per_frame(int(n), int(m)) for n, m in zip(N, M)], dtype=np.int64)
    sym_off = np.zeros(F + 1, dtype=np.int64)
    np.cumsum(L, out=sym_off[1:])
    cw_off = np.zeros(F + 1, dtype=np.int64)
    np.cumsum(N // 32, out=cw_off[1:])
    symbols = np.empty(int(sym_off[-1]), dtype=np.complex64)
    cw = np.empty(int(cw_off[-1]), dtype=np.uint32)
    is_hard = np.zeros(F, dtype=bool)
    is_hard[hard] = True
    easy = np.nonzero(~is_hard)[0]

    def gather(src, src_off, dst, dst_off, lengths):
        rel = np.arange(int(lengths.sum())) - np.repeat(np.cumsum(lengths) - lengths, lengths)
        dst[np.repeat(dst_off, lengths) + rel] = src[np.repeat(src_off, lengths) + rel]

    gather(mx["symbols"], mx["sym_offset"][easy], symbols, sym_off[easy], L[easy])
    gather(hx["symbols"], hx["sym_offset"], symbols, sym_off[hard], L[hard])
    gather(mx["codewords_packed"], mx["cw_offset"][easy], cw, cw_off[easy], (N[easy] // 32).astype(np.int64))
    gather(hx["codewords_packed"], hx["cw_offset"], cw, cw_off[hard], (N[hard] // 32).astype(np.int64))
    return {"hard": is_hard,"symbols": symbols, "N": N.astype(np.int32), "M": M.astype(np.int32), "L": L.astype(np.int32),
            "sym_offset": sym_off[:-1].copy(), "cw_offset": cw_off[:-1].copy(), "ebn0_db": snr,
            "codewords_packed": cw, "n_sym": int(sym_off[-1]), "n_cw_words": int(cw_off[-1])}


# -------------------------------------------------------------------------
# clocks during the timed region
# -------------------------------------------------------------------------
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "50"],
                                         stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except (OSError, ValueError):
            self.proc = None
            return
        # nvidia-smi's first query initialises NVML, which is slow and goes
        # through the driver: let it finish (its first sample written, at most
        # 3 s) before the measured work starts, so the two do not overlap
        t0 = time.time()
        while time.time() - t0 < 3.0 and self.proc.poll() is None:
            try:
                if os.path.getsize(self.path) > 0:
                    break
            except OSError:
                break
            time.sleep(0.01)

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        rows = []
        with open(self.path) as fh:
            for line in fh:
                t = [x.strip() for x in line.split(",")]
                if len(t) >= 9:
                    rows.append(t)
        os.unlink(self.path)
        if not rows:
            return None

        def num(x):
            try:
                return float(x)
            except ValueError:
                return None

        sm = [num(r[1]) for r in rows if num(r[1]) is not None]
        mx = [num(r[2]) for r in rows if num(r[2]) is not None]
        names = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")
        reasons = sorted({n for r in rows for n, v in zip(names, r[5:9]) if v.lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows)}


# -------------------------------------------------------------------------
# oracle (CPU baseline and the reference arm)
# -------------------------------------------------------------------------
def oracle_sample(cfg, inputs, per_snr, offset=0):
    """A bounded, SNR-stratified sample of the step's frames."""
    if cfg["kind"] == "mixed":
        idx = np.arange(offset, offset + per_snr * 3) % len(inputs["N"])
        return idx
    n_snr = len(cfg["snrs"])
    F = cfg["frames"]
    return np.concatenate([s * F + (offset + np.arange(per_snr)) % F for s in range(n_snr)])


def oracle_run(cfg, inputs, idx, threads):
    """Decode the sampled frames with the oracle; returns (useful checks, frames, seconds)."""
    import oracle

    t0 = time.perf_counter()
    useful = 0
    if cfg["kind"] == "mixed":
        for n in np.unique(inputs["N"][idx]):
            H = oracle.parity_H(int(n), int(n) // 2)
            for M in np.unique(inputs["M"][idx]):
                sel = idx[(inputs["N"][idx] == n) & (inputs["M"][idx] == M)]
                if sel.size == 0:
                    continue
                L = wl.symbols_per_frame(int(n), int(M))
                sym = np.stack([inputs["symbols"][inputs["sym_offset"][f]:inputs["sym_offset"][f] + L] for f in sel])
                r = oracle.decode_qam(H, sym, int(M), min(cfg["S"], L), cfg["cap"], threads=threads)
                useful += int(r["queries"].sum())
    else:
        H = oracle.parity_H(cfg["N"], cfg["K"])
        if cfg["kind"] == "ab":
            r = oracle.decode_ab(H, inputs["symbols"][idx], cfg["max_weight"], cfg["cap"], threads=threads)
        else:
            r = oracle.decode_qam(H, inputs["symbols"][idx], cfg["M"], cfg["S"], cfg["cap"], threads=threads)
        useful = int(r["queries"].sum())
    return useful, len(idx), time.perf_counter() - t0


def info_sets(cfg, source):
    if cfg["kind"] == "bler":
        return {}
    Ns = wl.MIXED_N if cfg["kind"] in ("mixed", "serve") else (cfg["N"],)
    out = {}
    for n in Ns:
        if source == "oracle":
            import oracle

            out[n] = oracle.info_set(n, n // 2)
        else:
            import paper_2405_01808_gb300 as g

            _, frozen = g.polar_H(n, n // 2)
            out[n] = np.setdiff1d(np.arange(n), frozen)
    return out


def run_reference(args, cfg):
    """The oracle as the reference arm: each step decodes a bounded sample."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    inputs = make_inputs(cfg, 0, info_sets(cfg, "oracle"))
    threads = os.cpu_count() or 1
    per = {"ab": 2000, "qam": 24, "mixed": 24}[cfg["kind"]]
    for w in range(args.warmup):
        oracle_run(cfg, inputs, oracle_sample(cfg, inputs, max(1, per // 8), offset=7 * w), threads)
    useful = frames = 0
    secs = 0.0
    for k in range(args.steps):
        u, f, s = oracle_run(cfg, inputs, oracle_sample(cfg, inputs, per, offset=per * k), threads)
        useful += u
        frames += f
        secs += s
    value = useful / secs
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "checks/s", "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * secs / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic (seeded random polar codewords over AWGN)",
        "config": {"workload": cfg["desc"], "sample_frames_per_step": frames // args.steps},
        "frames_per_s": frames / secs,
        "cpu_baseline": {"value": value, "unit": "checks/s", "cores": threads, "kind": "oracle",
                         "sample": f"{frames // args.steps} frames per step, SNR-stratified, of the workload"},
        "e2e": {"value": value, "unit": "checks/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


# -------------------------------------------------------------------------
# serving (continuous batching server, Poisson arrivals)
# -------------------------------------------------------------------------
def run_serving(args, cfg, g, inputs, resume_step=0):
    """Offer the requests at each Poisson rate; latency = completion - arrival.
    resume_step > 0: long frames leave their batch as device-resident cursors
    (grand_server_cfg.resume_weight_step)."""
    import torch

    codes = [g.Code.polar(n, n // 2) for n in wl.MIXED_N]
    code_of_N = {n: i for i, n in enumerate(wl.MIXED_N)}
    F = len(inputs["N"])
    sym = np.ascontiguousarray(inputs["symbols"])
    reqs = np.zeros(F, dtype=g.REQUEST_DTYPE)
    reqs["code"] = [code_of_N[int(n)] for n in inputs["N"]]
    reqs["M"] = inputs["M"]
    reqs["symbols"] = sym.ctypes.data + 8 * inputs["sym_offset"].astype(np.uint64)
    reqs["tag"] = np.arange(F, dtype=np.uint64)
    p = g.Params.make(M=0, S=cfg["S"], query_cap=cfg["cap"],
                      membership={"auto": 0, "hash": 3, "solve": 5}[args.membership])
    rows = []
    g_rng = np.random.default_rng(CONFIG_IDS["c5"])
    for rate in cfg["rates"]:
        srv = g.Server(codes, p, max_slots=1 << 18, max_device_bytes=1 << 30, max_batch=args.serve_batch,
                       n_streams=args.serve_streams, resume_weight_step=resume_step)
        # warm-up: a short burst (module load, pools)
        w = srv.submit(reqs[:20000])
        srv.drain(60.0)
        while len(srv.poll(1 << 16)):
            pass
        gaps = g_rng.exponential(1.0 / rate, size=F)
        offsets = np.cumsum(gaps * 1e9).astype(np.int64)
        # the first arrival lies 50 ms ahead: filling the arrival times of the
        # request table takes a few ms and must not start the stream late
        t0 = g.clock_ns() + 50_000_000
        arrival = t0 + offsets
        reqs["arrival_ns"] = arrival
        i = 0
        got = []
        submit_ns = np.zeros(F, dtype=np.int64)  # when the load generator handed each request over
        t_start = time.perf_counter()
        gc.disable()  # the load-generator loop stands in for a native client: no collector pauses inside it
        while i < F:
            now = g.clock_ns()
            j = int(np.searchsorted(arrival, now, side="right"))
            if j > i:
                k = srv.submit(reqs[i:j])
                submit_ns[i:i + k] = now
                i += k
            got.append(srv.poll(1 << 16))
            if time.perf_counter() - t_start > 120:
                break
        gc.enable()
        srv.drain(120.0)
        while True:
            tail = srv.poll(1 << 16)
            if not len(tail):
                break
            got.append(tail)
        st = srv.stats()
        srv.close()
        res = np.concatenate(got)
        warm = min(50000, F // 8)
        res = res[res["tag"] >= warm]  # the first requests warm the server at this rate
        lat_us = (res["done_ns"] - res["arrival_ns"]) / 1e3
        lag_us = (submit_ns[res["tag"].astype(np.int64)] - res["arrival_ns"]) / 1e3
        srv_us = lat_us - lag_us
        by_class = {}
        cont = res["continued"] == 1
        if cont.any():  # frames reported with their batch vs continued after it
            for name, m in (("with_batch", ~cont), ("continued", cont)):
                if m.any():
                    by_class[name] = {"requests": int(m.sum()), "p50": float(np.percentile(lat_us[m], 50)),
                                      "p99": float(np.percentile(lat_us[m], 99)), "max": float(lat_us[m].max())}
        if "hard" in inputs:  # latency of the injected long frames and of the rest, separately
            hmask = inputs["hard"][res["tag"].astype(np.int64)]
            for name, m in (("regular", ~hmask), ("hard", hmask)):
                if m.any():
                    by_class[name] = {"requests": int(m.sum()), "p50": float(np.percentile(lat_us[m], 50)),
                                      "p99": float(np.percentile(lat_us[m], 99)), "max": float(lat_us[m].max()),
                                      "server_p50": float(np.percentile(srv_us[m], 50)),
                                      "server_p99": float(np.percentile(srv_us[m], 99))}
        span = (res["done_ns"].max() - arrival[warm]) / 1e9
        rows.append({"offered_frames_per_s": rate, "completed": int(len(res)),
                     "frames_per_s": len(res) / span, "checks_per_s": float(res["queries"].sum()) / span,
                     "latency_us": {"p50": float(np.percentile(lat_us, 50)), "p99": float(np.percentile(lat_us, 99)),
                                    "max": float(lat_us.max())},
                     "batches": st["batches"], "mean_batch": st["batched_frames"] / max(1, st["batches"]),
                     "max_inflight_batches": st["max_inflight_batches"], "rejected_submits": st["rejected"],
                     "batch_service_us": {"mean": st["batch_service_ns"] / max(1, st["batches"]) / 1e3,
                                          "max": st["max_batch_service_ns"] / 1e3},
                     "launch_us": {"mean": st["launch_ns"] / max(1, st["batches"]) / 1e3,
                                   "max": st["max_launch_ns"] / 1e3},
                     "latency_us_hist": np.percentile(lat_us, [10, 25, 50, 75, 90, 95, 99, 99.9]).round(1).tolist(),
                     # the two parts: the load generator's delay in handing requests over, and the server's time
                     "client_lag_us": {"p50": float(np.percentile(lag_us, 50)), "p99": float(np.percentile(lag_us, 99)),
                                       "max": float(lag_us.max())},
                     "server_latency_us": {"p50": float(np.percentile(srv_us, 50)),
                                           "p99": float(np.percentile(srv_us, 99)), "max": float(srv_us.max())},
                     "errors": st["errors"], "resume_weight_step": resume_step, "latency_us_by_class": by_class,
                     "long_frames": st["long_frames"], "resume_launches": st["resume_launches"]})
    last = res
    # the plain one-frame-per-launch GPU path on a sample of the same requests:
    # per request the host->device copy of its symbols, one decode call and the
    # read-back of its result, one request after another (no batching); its
    # outputs must equal the server's for the same requests (same BLER)
    n_one = min(2000, F)
    pick = np.linspace(min(min(50000, F // 8), F - 1), F - 1, n_one).astype(np.int64)
    pos = np.full(F, -1, dtype=np.int64)
    pos[last["tag"].astype(np.int64)] = np.arange(len(last))
    params_of_M = {}
    lat_one = np.zeros(n_one)
    equal = True
    torch.cuda.synchronize()
    t_all = time.perf_counter()
    for k, f in enumerate(pick.tolist()):
        n, M = int(inputs["N"][f]), int(inputs["M"][f])
        L = wl.symbols_per_frame(n, M)
        o = int(inputs["sym_offset"][f])
        if M not in params_of_M:
            params_of_M[M] = g.Params.make(M=M, S=cfg["S"], query_cap=cfg["cap"], membership=p.membership)
        t1 = time.perf_counter()
        x = torch.from_numpy(sym[o:o + L].reshape(1, L)).cuda()
        r = g.decode_symbols(codes[code_of_N[n]], params_of_M[M], x)
        cw_h, q_h, ab_h = r["cw"].cpu().numpy().view(np.uint32), r["queries"].cpu().numpy(), r["abandon"].cpu().numpy()
        lat_one[k] = time.perf_counter() - t1
        j = pos[f]
        if j >= 0:
            row = last[j]
            equal &= bool(int(row["queries"]) == int(q_h[0]) and int(row["abandon"]) == int(ab_h[0])
                          and np.array_equal(row["cw"][:n // 32], cw_h[0]))
    span_one = time.perf_counter() - t_all
    for c in codes:
        c.close()
    one = {"frames_per_s": n_one / span_one,
           "latency_us": {"p50": float(np.percentile(lat_one, 50) * 1e6), "p99": float(np.percentile(lat_one, 99) * 1e6)},
           "outputs_equal_server": equal,
           "sample": f"{n_one} requests spread over the stream, each copied in, decoded by its own call and read back",
           "note": "its frames/s is the most the plain path can serve; an offered rate above it queues without bound"}
    return rows, one


# -------------------------------------------------------------------------
# BLER sweep (the paper's experiment, Sec. IV / Fig. 4, with this decoder)
# -------------------------------------------------------------------------
BLER_GRID = {4: range(0, 9), 16: range(4, 13), 64: range(8, 17), 256: range(12, 21), 1024: range(16, 25),
             4096: range(20, 29)}


def run_bler(args, cfg, g):
    """BLER per (N, M, Eb/N0) at S=8: frames generated on the device in chunks
    (torch transmitter of `workloads`, seeded per point), decoded by the fused
    call, compared with the sent codewords on the device."""
    import torch

    rows = []
    frames = cfg["frames"]
    chunk = min(frames, 250000)
    dec_s = 0.0
    n_total = 0
    dev = torch.device("cuda", torch.cuda.current_device())
    for N in wl.MIXED_N:
        H, frozen = g.polar_H(N, N // 2)
        info = np.setdiff1d(np.arange(N), frozen)
        code = g.Code(H, N, N // 2)
        for M, grid in BLER_GRID.items():
            p = g.Params.make(M=M, S=cfg["S"], query_cap=4 ** cfg["S"])
            curve = []
            for snr in grid:
                n_err = n_ab = n_und = 0
                q_sum = 0.0
                for c0 in range(0, frames, chunk):
                    F = min(chunk, frames - c0)
                    seed = (CONFIG_IDS["bler"] << 40) ^ (N << 28) ^ (M << 12) ^ (int(snr) << 6) ^ (c0 // chunk)
                    d = wl.torch_qam_frames(seed, F, N, info, M, float(snr), dev)
                    torch.cuda.synchronize()
                    t0 = time.perf_counter()
                    r = g.decode_symbols(code, p, d["symbols"])
                    torch.cuda.synchronize()
                    dec_s += time.perf_counter() - t0
                    n_total += F
                    err = (r["cw"] != d["codewords_packed"].view(r["cw"].dtype)).any(dim=1)
                    ab = r["abandon"] == 1
                    n_err += int(err.sum().item())
                    n_ab += int(ab.sum().item())
                    n_und += int((err & ~ab).sum().item())
                    q_sum += float(r["queries"].to(torch.float64).sum().item())
                curve.append({"ebn0_db": snr, "bler": n_err / frames, "abandon": n_ab / frames,
                              "undetected": n_und / frames, "mean_queries": q_sum / frames})
            rows.append({"N": N, "M": M, "L": wl.symbols_per_frame(N, M), "curve": curve})
        code.close()
    return rows, n_total / dec_s


def _c2_like_batch(cfg, g):
    """The N=128 16-QAM frames of the default workload (same seeds), on the device."""
    import torch

    H, frozen = g.polar_H(cfg["N"], cfg["K"])
    info = np.setdiff1d(np.arange(cfg["N"]), frozen)
    parts = [wl.qam_frames(CONFIG_IDS[cfg["name"]], i, cfg["frames"], cfg["N"], info, cfg["M"], snr)
             for i, snr in enumerate(cfg["snrs"])]
    sym = torch.from_numpy(np.concatenate([p["symbols"] for p in parts])).cuda()
    cwt = np.concatenate([p["codewords_packed"] for p in parts])
    return g.Code(H, cfg["N"], cfg["K"]), sym, cwt


def _timed_decode(g, code, p, sym):
    import torch

    torch.cuda.synchronize()
    t0 = time.perf_counter()
    r = g.decode_symbols(code, p, sym, stats=True)
    torch.cuda.synchronize()
    return r, time.perf_counter() - t0


def run_orders(args, cfg, g):
    """Query counts and BLER of the TEP orders on the same frames (one decode
    per order and setting, after a warm-up call)."""
    code, sym, cwt = _c2_like_batch(cfg, g)
    F = cfg["frames"]
    variants = [("paper (Def. III.1/III.2)", g.ORDER_QAM_NNE, g.LIK_THRESHOLD),
                ("paper, literal Def. III.1 edge distance", g.ORDER_QAM_NNE, g.LIK_LITERAL),
                ("nearer axis first", g.ORDER_QAM_NEARER, g.LIK_THRESHOLD),
                ("five-point NNE (4 alternatives, no diagonal)", g.ORDER_QAM_NNE5, g.LIK_THRESHOLD)]
    rows = []
    for S, cap_of in ((8, lambda o: (5 if o == g.ORDER_QAM_NNE5 else 4) ** 8), (10, lambda o: 1 << 20)):
        for name, order, lik in variants:
            p = g.Params.make(order=order, M=cfg["M"], S=S, query_cap=cap_of(order), lik_variant=lik)
            _timed_decode(g, code, p, sym[:1000])
            r, secs = _timed_decode(g, code, p, sym)
            cw = r["cw"].cpu().numpy().view(np.uint32)
            q = r["queries"].cpu().numpy().view(np.uint32).astype(np.int64)
            ab = r["abandon"].cpu().numpy()
            per_snr = []
            for i, snr in enumerate(cfg["snrs"]):
                sl = slice(i * F, (i + 1) * F)
                err = (cw[sl] != cwt[sl]).any(axis=1)
                dec = ab[sl] == 0
                per_snr.append({"ebn0_db": snr, "bler": float(err.mean()), "abandon": float((ab[sl] == 1).mean()),
                                "undetected": float((err & dec).mean()), "mean_queries": float(q[sl].mean()),
                                "mean_queries_decoded": float(q[sl][dec].mean()) if dec.any() else None,
                                "median_queries_correct": float(np.median(q[sl][dec & ~err])) if (dec & ~err).any()
                                else None})
            rows.append({"order": name, "S": S, "cap": cap_of(order), "seconds": secs,
                         "frames_per_s": len(q) / secs, "useful_checks_per_s": float(q.sum()) / secs,
                         "per_snr": per_snr})
    code.close()
    return rows


def run_membership(args, cfg, g):
    """Device time of the three membership tests on the same frames."""
    code, sym, cwt = _c2_like_batch(cfg, g)
    rows = []
    ref = None
    for name, mem in (("split search, syndrome deltas (bit-sliced)", g.MEMBERSHIP_AUTO),
                      ("per-TEP syndrome deltas", g.MEMBERSHIP_DELTA),
                      ("per-TEP row parity (Alg. 1 product)", g.MEMBERSHIP_ROW_PARITY),
                      ("hash join of the split (decision, no per-TEP test)", g.MEMBERSHIP_HASH)):
        p = g.Params.make(M=cfg["M"], S=cfg["S"], query_cap=cfg["cap"], membership=mem)
        _timed_decode(g, code, p, sym[:2000])
        r, secs = _timed_decode(g, code, p, sym)
        q = r["queries"].cpu().numpy().view(np.uint32).astype(np.int64)
        out = (r["cw"].cpu().numpy(), q, r["abandon"].cpu().numpy())
        same = True if ref is None else all(np.array_equal(a, b) for a, b in zip(out, ref))
        ref = ref or out
        kern_ms = float(r["prep_ms"] + r["search_ms"])
        rows.append({"membership": name, "seconds": secs, "kernel_ms": kern_ms,
                     "useful_checks_per_s": float(q.sum()) / (kern_ms / 1e3),
                     "evaluated_checks": int(r["evaluated_checks"]),
                     "evaluated_checks_per_s": r["evaluated_checks"] / (kern_ms / 1e3),
                     "results_equal_split_search": bool(same)})
    # the default workload's whole batch (300,000 frames): split search against the hash join
    full = dict(cfg, frames=100000)
    code2, sym2, _ = _c2_like_batch(full, g)
    base = None
    for name, mem in (("split search (default)", g.MEMBERSHIP_AUTO), ("hash join", g.MEMBERSHIP_HASH)):
        p = g.Params.make(M=cfg["M"], S=cfg["S"], query_cap=cfg["cap"], membership=mem)
        _timed_decode(g, code2, p, sym2)
        ms = []
        for _ in range(5):
            r, _secs = _timed_decode(g, code2, p, sym2)
            ms.append(float(r["prep_ms"] + r["search_ms"]))
        q = r["queries"].cpu().numpy().view(np.uint32).astype(np.int64)
        out = (r["cw"].cpu().numpy(), q, r["abandon"].cpu().numpy())
        same = True if base is None else all(np.array_equal(x, y) for x, y in zip(out, base))
        base = base or out
        rows.append({"membership": name + ", 300,000-frame batch", "kernel_ms": statistics.median(ms),
                     "search_ms": float(r["search_ms"]), "frames_per_s": len(q) / (statistics.median(ms) / 1e3),
                     "useful_checks_per_s": float(q.sum()) / (statistics.median(ms) / 1e3),
                     "evaluated_checks": int(r["evaluated_checks"]), "results_equal_split_search": bool(same)})
    code2.close()
    code.close()
    return rows


# -------------------------------------------------------------------------
# GPU arm
# -------------------------------------------------------------------------
def run_config(args, cfg, g, ctx):
    """One workload as the bench line's record: device-timed decode steps
    (inputs resident, L2 flushed), the kernel split and roofline, the hash
    join on the same batch, the public demodulation, the host-memory (e2e)
    call, the one-frame-per-launch path and the oracle on a bounded sample.
    Returns the record on rank 0 (None elsewhere)."""
    import torch

    rank, world, dist, local = ctx["rank"], ctx["world"], ctx["dist"], ctx["local"]
    tiles = tuple(int(t) for t in args.tiles.split(","))
    membership = {"auto": 0, "hash": 3}[args.membership]
    info = info_sets(cfg, "library")
    inputs = make_inputs(cfg, rank, info)
    dev = torch.device("cuda", local)
    stream = torch.cuda.current_stream()
    # ---- code objects and device buffers
    if cfg["kind"] == "mixed":
        codes = [g.Code.polar(n, n // 2) for n in wl.MIXED_N]
        desc = g.frame_desc(np.searchsorted(np.array(wl.MIXED_N), inputs["N"]), inputs["M"], inputs["sym_offset"],
                            inputs["cw_offset"])
        d_desc = torch.from_numpy(desc.view(np.uint8)).to(dev)
        n_frames = len(inputs["N"])
        n_cw = inputs["n_cw_words"]
        p = g.Params.make(M=0, S=cfg["S"], query_cap=cfg["cap"], tiles=tiles, membership=membership)
        alg_words = None
    else:
        codes = [g.Code.polar(cfg["N"], cfg["K"])]
        n_frames = len(inputs["symbols"])
        n_cw = n_frames * cfg["N"] // 32
        if cfg["kind"] == "ab":
            p = g.Params.make(order=g.ORDER_HAMMING, M=2, max_weight=cfg["max_weight"], query_cap=cfg["cap"])
        else:
            p = g.Params.make(M=cfg["M"], S=cfg["S"], query_cap=cfg["cap"], tiles=tiles, membership=membership)
        alg_words = (cfg["N"] - cfg["K"]) / 32.0
    h_sym = torch.from_numpy(inputs["symbols"]).pin_memory()
    d_sym = h_sym.to(dev)
    d_cw = torch.empty(n_cw, dtype=torch.int32, device=dev)
    d_q = torch.empty(n_frames, dtype=torch.int32, device=dev)
    d_ab = torch.empty(n_frames, dtype=torch.uint8, device=dev)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)

    tune = None
    plan = None
    if cfg["kind"] == "qam" and not any(tiles):
        # launch shapes from the autotuner on frames spread over the batch
        # (every SNR point); the outputs do not depend on them
        n_tune = min(n_frames, 100000)
        pick = torch.from_numpy(np.linspace(0, n_frames - 1, n_tune).astype(np.int64)).to(dev)
        tune = g.autotune(codes[0], p, d_sym.index_select(0, pick))
    if cfg["kind"] == "mixed":
        # tiles from the autotuner on a 100,000-frame sample, then the whole
        # batch captured once into a CUDA graph (one replay per step)
        n_tune = min(n_frames, 100000)
        tune = g.autotune_mixed(codes, p, d_desc[: n_tune * g.FRAME_DESC_DTYPE.itemsize], d_sym, n_cw)
        plan = g.plan_mixed(codes, p, d_desc, d_sym, d_cw, d_q, d_ab)

    if cfg["kind"] != "mixed":
        # the whole decode call captured once into a CUDA graph (one replay per
        # timed step: no host-side launch overhead inside the device-timed step)
        plan = g.plan_symbols(codes[0], p, d_sym, d_cw.view(n_frames, -1), d_q, d_ab)

    def step(sym, stats=True):
        if sym is d_sym and not stats:
            plan.launch()
            return None
        if cfg["kind"] == "mixed":
            return g.decode_mixed(codes, p, d_desc, sym, n_cw, cw=d_cw, queries=d_q, abandon=d_ab, stats=stats)
        cw2 = d_cw.view(n_frames, -1)
        return g.decode_symbols(codes[0], p, sym, cw=cw2, queries=d_q, abandon=d_ab, stats=stats)

    for _ in range(args.warmup):
        step(d_sym, stats=False)
    torch.cuda.synchronize()

    # ---- timed steps (device-resident inputs)
    clocks = ClockSampler(local)
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    clocks.start()
    step_ms, search_ms, prep_ms = [], [], []
    useful_total = 0
    search_useful = 0
    evaluated = 0
    hard = 0
    graph_steps = True  # every workload replays its CUDA-graph plan
    split_after = True  # kernel split and counters from one direct call after the timed steps
    for _ in range(args.steps):
        flush.zero_()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        # the graph replay and the one-kernel GRAND-AB step run without statistics (asynchronous)
        r = step(d_sym, stats=not split_after)
        e1.record(stream)
        e1.synchronize()
        step_ms.append(e0.elapsed_time(e1))
        if r is not None and "search_ms" in r:
            search_ms.append(r["search_ms"])
            prep_ms.append(r["prep_ms"])
            search_useful += r["search_useful"]
            evaluated += r["evaluated_checks"]
            hard += r["hard_frames"]
        useful_total += int(d_q.to(torch.int64).sum().item())  # outside the events
    if split_after:  # kernel split and counters from one direct call of the same batch
        flush.zero_()
        r = step(d_sym, stats=True)
        search_ms, prep_ms = [r["search_ms"]], [r["prep_ms"]]
        search_useful, evaluated, hard = (r["search_useful"] * args.steps, r["evaluated_checks"] * args.steps,
                                          r["hard_frames"] * args.steps)
        if cfg["kind"] == "ab":  # one kernel answers every query
            search_useful = useful_total
    torch.cuda.synchronize()
    clk = clocks.stop()
    total_ms = sum(step_ms)
    from paper_2405_01808_gb300 import dist as gdist

    (useful_all, frames_all), tmax_ms = gdist.aggregate([useful_total, n_frames * args.steps], total_ms,
                                                        dist, device=dev)
    if dist:
        dist.barrier()
    value = useful_all / (tmax_ms / 1e3)
    frames_per_s = frames_all / (tmax_ms / 1e3)

    # ---- correctness of the timed output (decoded words vs transmitted)
    cw_host = d_cw.cpu().numpy().view(np.uint32)
    ab_host = d_ab.cpu().numpy()
    if cfg["kind"] == "mixed":
        sent = inputs["codewords_packed"]
        errs = 0
        for f in range(0, n_frames, max(1, n_frames // 20000)):
            o, n = inputs["cw_offset"][f], inputs["N"][f] // 32
            errs += int(not np.array_equal(cw_host[o:o + n], sent[o:o + n]))
        bler = errs / len(range(0, n_frames, max(1, n_frames // 20000)))
    else:
        bler = float(np.mean((cw_host.reshape(n_frames, -1) != inputs["codewords_packed"]).any(axis=1)))

    # ---- the public demodulation call (Def. III.1/III.2 alone, grand_demod) on the
    #      same symbols: HBM-bound, measured against the copy bandwidth
    demod = None
    if cfg["kind"] == "qam":
        L = inputs["symbols"].shape[1]
        dm_out = g.demod(d_sym, cfg["M"], cfg["N"])
        # calls back to back over rotating copies of the symbols: each call
        # reads a batch the previous calls evicted from L2 (the rotation holds
        # 4 x the batch plus the outputs, far more than L2), and the GPU never
        # idles between the events while the host issues the next call
        rot = [d_sym] + [d_sym.clone() for _ in range(3)]
        per_step = 8
        for k in range(args.warmup):
            g.demod(rot[k % 4], cfg["M"], cfg["N"], outputs=dm_out)
        dm_ms = []
        for _ in range(args.steps):
            flush.zero_()
            gpu_busy_us(100)
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            for k in range(per_step):
                g.demod(rot[k % 4], cfg["M"], cfg["N"], outputs=dm_out)
            e1.record(stream)
            e1.synchronize()
            dm_ms.append(e0.elapsed_time(e1) / per_step)
        del rot
        # symbols in (8 B), hard index, key, mask, likelihood out (2 + 4 + 1 + 4 B), hard word out
        dm_bytes = n_frames * L * (8 + 11) + n_frames * cfg["N"] // 8
        peak, src = hbm_peak()
        ach = dm_bytes / (statistics.mean(dm_ms) / 1e3) / 1e9
        demod = {"kernel": "k_demod", "bound": "hbm", "ms": statistics.mean(dm_ms), "bytes": dm_bytes,
                 "achieved": ach, "peak": peak, "unit": "GB/s", "frac": ach / peak, "peak_source": src,
                 "timing": "CUDA events around 8 calls back to back on 4 rotating copies of the batch (each "
                           "call's symbols evicted from L2 by the others); per-call mean"}

    # ---- the fastest exact decode of the same batch: the autotuner chooses
    #      between the TEP-by-TEP split search and the hash join of the split
    #      (GRAND_MEMBERSHIP_FASTEST; identical outputs) and their launch
    #      shapes; frames/s and latency on the chosen path (a CUDA-graph plan
    #      for the uneven batch), reported beside the checks/s headline
    fastest = None
    if cfg["kind"] in ("qam", "mixed") and args.membership == "auto":
        ref_out = (d_cw.clone(), d_q.clone(), d_ab.clone())
        pf = g.Params.make(order=p.order, M=p.M, S=p.S, query_cap=p.query_cap, membership=g.MEMBERSHIP_FASTEST)
        n_tune = min(n_frames, 100000)
        if cfg["kind"] == "mixed":
            ftune = g.autotune_mixed(codes, pf, d_desc[: n_tune * g.FRAME_DESC_DTYPE.itemsize], d_sym, n_cw)
            fplan = g.plan_mixed(codes, pf, d_desc, d_sym, d_cw, d_q, d_ab)
            fstep = fplan.launch
        else:
            # the tuning sample: frames spread over the batch (every SNR point)
            pick = torch.from_numpy(np.linspace(0, n_frames - 1, n_tune).astype(np.int64)).to(dev)
            ftune = g.autotune(codes[0], pf, d_sym.index_select(0, pick))
            fplan = None

            def fstep():
                g.decode_symbols(codes[0], pf, d_sym, cw=d_cw.view(n_frames, -1), queries=d_q, abandon=d_ab)

        for _ in range(args.warmup):
            fstep()
        f_ms = []
        for _ in range(args.steps):
            flush.zero_()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            fstep()
            e1.record(stream)
            e1.synchronize()
            f_ms.append(e0.elapsed_time(e1))
        same = all(torch.equal(x, y) for x, y in zip((d_cw, d_q, d_ab), ref_out))
        if fplan is not None:
            fplan.close()
        fastest = {"membership": {0: "split search (TEP by TEP)", 3: "hash join"}.get(ftune["membership"]),
                   "tiles": list(ftune["tiles"]), "ms_per_step": statistics.mean(f_ms),
                   "frames_per_s": n_frames / (statistics.mean(f_ms) / 1e3),
                   "latency_ms": {"p50": float(np.percentile(f_ms, 50)), "p99": float(np.percentile(f_ms, 99))},
                   "outputs_equal": bool(same), "graph": cfg["kind"] == "mixed",
                   "what": "the autotuner's fastest exact membership test (GRAND_MEMBERSHIP_FASTEST) on the same "
                           "batch: same outputs; a hash join decides the queries without testing them one by "
                           "one, so this line reports frames/s, not checks"}

    # ---- the same batch through GRAND_MEMBERSHIP_SOLVE: the first hit by
    #      Gaussian elimination over each frame's TEP coordinates (the TEP
    #      space of S' ranks with at most 4 alternatives is a GF(2) coordinate
    #      space, so its codewords are the solutions of a linear system), one
    #      CUDA-graph replay per step like the headline; identical outputs.
    #      It tests no TEP one by one, so it reports frames/s, not checks.
    solve = None
    if cfg["kind"] in ("qam", "mixed") and args.membership == "auto":
        try:
            ref_out = (d_cw.clone(), d_q.clone(), d_ab.clone())
            ps = g.Params.make(order=p.order, M=p.M, S=p.S, query_cap=p.query_cap, membership=g.MEMBERSHIP_SOLVE)
            if cfg["kind"] == "mixed":
                splan = g.plan_mixed(codes, ps, d_desc, d_sym, d_cw, d_q, d_ab)
                rs = g.decode_mixed(codes, ps, d_desc, d_sym, n_cw, cw=d_cw, queries=d_q, abandon=d_ab, stats=True)
            else:
                splan = g.plan_symbols(codes[0], ps, d_sym, d_cw.view(n_frames, -1), d_q, d_ab)
                rs = g.decode_symbols(codes[0], ps, d_sym, cw=d_cw.view(n_frames, -1), queries=d_q, abandon=d_ab,
                                      stats=True)
            for _ in range(args.warmup):
                splan.launch()
            s_ms = []
            for _ in range(args.steps):
                flush.zero_()
                e0 = torch.cuda.Event(enable_timing=True)
                e1 = torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                splan.launch()
                e1.record(stream)
                e1.synchronize()
                s_ms.append(e0.elapsed_time(e1))
            same = all(torch.equal(x, y) for x, y in zip((d_cw, d_q, d_ab), ref_out))
            splan.close()
            s_mean = statistics.mean(s_ms)
            solve = {"membership": "linear solve (GRAND_MEMBERSHIP_SOLVE)", "ms_per_step": s_mean,
                     "frames_per_s": n_frames / (s_mean / 1e3),
                     "latency_ms": {"p50": float(np.percentile(s_ms, 50)), "p99": float(np.percentile(s_ms, 99))},
                     "kernel_ms": {"prep": rs["prep_ms"], "search": rs["search_ms"]},
                     "frames_to_tep_search": int(rs["hard_frames"]), "ranked_solutions": int(rs["evaluated_checks"]),
                     "outputs_equal": bool(same), "graph": True, "profile": "profiles/k_prep_solve_c2_small.md",
                     "what": "the same batch with the first hit found by Gaussian elimination over each frame's TEP "
                             "coordinates (the codewords of the TEP space are the solutions of a GF(2) linear "
                             "system; the first hit is the one of smallest canonical rank): same outputs, no TEP "
                             "tested one by one, so this line reports frames/s, not checks"}
        except g.GrandError as e:  # an auxiliary leg: report it, keep the headline
            solve = {"membership": "linear solve (GRAND_MEMBERSHIP_SOLVE)", "error": str(e)}

    # ---- e2e: the same decode from pinned host buffers, copies in the timed
    #      region, through the library's host-memory calls
    #      (grand_decode_symbols_host / grand_decode_mixed_host: chunks on two
    #      streams, copies overlapped with decoding).
    h_cw = torch.empty(n_cw, dtype=torch.int32).pin_memory()
    h_q = torch.empty(n_frames, dtype=torch.int32).pin_memory()
    h_ab = torch.empty(n_frames, dtype=torch.uint8).pin_memory()
    d_sym2 = torch.empty_like(d_sym)
    host_api = cfg["kind"] in ("qam", "ab", "mixed")
    if cfg["kind"] == "mixed":  # the descriptors are host input too, page-locked like the symbols
        h_desc = torch.from_numpy(desc.view(np.uint8)).pin_memory()
    e2e_ms = []
    for it in range(1 + max(2, min(args.steps, 5))):  # the first call is untimed (pool growth, streams)
        flush.zero_()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        if host_api and cfg["kind"] == "mixed":
            g.decode_mixed_host(codes, p, h_desc, h_sym, n_cw, cw=h_cw, queries=h_q, abandon=h_ab, stream=stream)
        elif host_api:
            g.decode_symbols_host(codes[0], p, h_sym, cw=h_cw, queries=h_q, abandon=h_ab, stream=stream)
        else:
            d_sym2.copy_(h_sym, non_blocking=True)
            step(d_sym2, stats=False)
            h_cw.copy_(d_cw, non_blocking=True)
            h_q.copy_(d_q, non_blocking=True)
            h_ab.copy_(d_ab, non_blocking=True)
        e1.record(stream)
        e1.synchronize()
        if it:
            e2e_ms.append(e0.elapsed_time(e1))
    e2e_value = (useful_total / args.steps) / (statistics.mean(e2e_ms) / 1e3)
    e2e_equal = bool(torch.equal(h_cw, d_cw.cpu()) and torch.equal(h_q, d_q.cpu()) and torch.equal(h_ab, d_ab.cpu()))

    # ---- the plain one-frame-per-launch GPU path on a sample (same frames, same results)
    one = None
    if cfg["kind"] in ("qam", "mixed"):
        # S' = 12 frames that abandon run 2^24 queries each in one warp: a smaller sample
        n_one = min(2000 if cfg.get("S", 10) <= 10 else 200, n_frames)
        idx = np.linspace(0, n_frames - 1, n_one).astype(np.int64)
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for f in idx.tolist():
            if cfg["kind"] == "mixed":
                dsz = g.FRAME_DESC_DTYPE.itemsize
                g.decode_mixed(codes, p, d_desc[f * dsz:(f + 1) * dsz], d_sym, n_cw, cw=d_cw, queries=d_q[f:f + 1],
                               abandon=d_ab[f:f + 1])
            else:
                g.decode_symbols(codes[0], p, d_sym[f:f + 1], cw=d_cw.view(n_frames, -1)[f:f + 1],
                                 queries=d_q[f:f + 1], abandon=d_ab[f:f + 1])
        e1.record(stream)
        e1.synchronize()
        one_ms = e0.elapsed_time(e1)
        one = {"frames_per_s": n_one / (one_ms / 1e3), "ms_per_frame": one_ms / n_one,
               "sample": f"{n_one} frames evenly spread over the batch, one decode call each"}

    # ---- roofline of the dominant kernel (the TEP search)
    roofline = None
    if sum(search_ms) > 0 and args.membership == "auto":  # TEPs tested one by one
        roofline = search_roofline(cfg, evaluated / args.steps, search_useful / args.steps, hard / args.steps,
                                   statistics.mean(search_ms), alg_words, frames=n_frames)

    # ---- CPU baseline: the oracle on a bounded sample (rank 0, N=1)
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        # frames per SNR point (a 2^24-query abandon of the S=12 workloads costs
        # the oracle 15-25 s of one core, so those take one frame per point
        # and no single-core leg)
        per, per1 = {"ab": (3000, 750), "qam": (48, 12), "mixed": (40, 10)}[cfg["kind"]]
        if cfg["kind"] == "qam" and cfg["S"] > 10:
            per, per1 = 1, 0
        idx = oracle_sample(cfg, inputs, per)
        threads = os.cpu_count() or 1
        u, f, s = oracle_run(cfg, inputs, idx, threads)
        cpu = {"value": u / s, "unit": "checks/s", "cores": min(threads, f), "kind": "oracle",
               "sample": f"{f} frames ({per} per SNR point) of the same workload", "frames_per_s": f / s,
               "seconds": s}
        # the same oracle on one core, on a quarter of that sample
        if per1:
            idx1 = oracle_sample(cfg, inputs, per1)
            u1, f1, s1 = oracle_run(cfg, inputs, idx1, 1)
            cpu["single_core"] = {"value": u1 / s1, "unit": "checks/s", "frames": f1, "seconds": s1,
                                  "frames_per_s": f1 / s1}

    if plan is not None:
        plan.close()
    line = None
    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": "checks/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": tmax_ms / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "u32",
            "data": "synthetic (seeded random polar codewords over AWGN)",
            "config": {"workload": cfg["desc"], "frames_per_step_per_gpu": n_frames, "tiles": list(p.tiles),
                       "l2": "flushed before every timed step (256 MiB write)",
                       "membership": args.membership,
                       "parallelism": f"frames sharded, {world} replica(s)"},
            "frames_per_s": frames_per_s,
            "latency_ms": {"p50": float(np.percentile(step_ms, 50)), "p99": float(np.percentile(step_ms, 99)),
                           "what": "whole-batch decode time per step"},
            "bler": bler,
            "evaluated_checks_per_step": evaluated / args.steps,
            "useful_checks_per_step": useful_total / args.steps,
            "hard_frames_per_step": hard / args.steps,
            "kernel_ms": ({"prep": statistics.mean(prep_ms), "search": statistics.mean(search_ms)} if search_ms
                          else None),
            "roofline": roofline,
            "fastest_exact": fastest,
            "solve": solve,
            "demod": demod,
            "one_frame_per_launch": one,
            "autotune": tune,
            "cpu_baseline": cpu,
            "e2e": {"value": e2e_value, "unit": "checks/s", "h2d_bytes_per_step": int(h_sym.numel() * h_sym.element_size()),
                    "d2h_bytes_per_step": int(n_cw * 4 + n_frames * 5), "ms_per_step": statistics.mean(e2e_ms),
                    "api": ("grand_decode_mixed_host" if cfg["kind"] == "mixed" else "grand_decode_symbols_host")
                           + " (chunks on two streams, copies overlapped with decoding)",
                    "outputs_equal_device": e2e_equal},
            "gpu_launches": 2 * args.steps if cfg["kind"] != "ab" else args.steps,
            "graph": bool(graph_steps),
            "clocks": clk,
        }
    return line


def run_serve_config(args, cfg, g, ctx):
    """The serving workload as a bench record: Poisson arrivals at each rate
    through the continuous-batching server (frames/s, p50/p99 latency), and
    the plain one-frame-per-launch path on a sample of the same requests. The
    adversarial mix runs twice: long frames whole inside their batch, then
    carried as device-resident cursors (resume_weight_step)."""
    rank, world, local = ctx["rank"], ctx["world"], ctx["local"]
    inputs = make_inputs(cfg, rank, info_sets(cfg, "library"))
    clocks = ClockSampler(local)
    clocks.start()
    rows, one = run_serving(args, cfg, g, inputs, resume_step=0 if cfg.get("adversarial") else args.serve_resume_step)
    carried = None
    if cfg.get("adversarial") and args.membership != "solve":
        carried, _ = run_serving(args, cfg, g, inputs, resume_step=max(1, args.serve_resume_step))
    clk = clocks.stop()
    if rank != 0:
        return None
    head = (carried or rows)[-1]
    line = {"metric": METRIC, "value": head["frames_per_s"], "unit": "frames/s", "n_gpus": world,
            "steps": len(rows), "warmup": 1, "ms_per_step": None, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "u32",
            "data": "synthetic (seeded random polar codewords over AWGN)",
            "config": {"workload": cfg["desc"], "requests_per_rate": len(inputs["N"]),
                       "server": f"max_slots 262144, budget 1 GiB, max_batch {args.serve_batch}, "
                                 f"{args.serve_streams} streams",
                       "membership": {"auto": "split search (TEP by TEP)", "hash": "hash join",
                                      "solve": "linear solve (GRAND_MEMBERSHIP_SOLVE)"}[args.membership]},
            "latency_us": head["latency_us"], "rates": rows, "one_frame_per_launch": one, "clocks": clk,
            "e2e": {"value": head["frames_per_s"], "unit": "frames/s",
                    "h2d_bytes_per_step": int(inputs["symbols"].nbytes),
                    "d2h_bytes_per_step": int(len(inputs["N"]) * 160)},
            "gpu_launches": int(sum(r["batches"] for r in rows + (carried or [])) * 2)}
    if carried is not None:
        line["rates_long_frames_carried"] = carried
    return line


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gpu", choices=("gpu", "reference"))
    ap.add_argument("--config", default=None, choices=sorted(CONFIGS),
                    help="one workload alone (default: the N=128 16-QAM headline with the other throughput "
                         "workloads as sub-records)")
    ap.add_argument("--subconfigs", default="c1,c3a,c3b,c4,c5",
                    help="workloads measured after the headline in the default run")
    ap.add_argument("--no-subconfigs", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--frames", type=int, default=0, help="override frames per SNR (for quick runs)")
    ap.add_argument("--tiles", default="0,0,0,0", help="launch shape (grand_params.tiles), 0 = automatic")
    ap.add_argument("--membership", default="auto", choices=("auto", "hash", "solve"),
                    help="membership test of the search (the headline uses the TEP-by-TEP search; "
                         "solve: serving configs only -- the other records carry it under 'solve')")
    ap.add_argument("--serve-batch", type=int, default=65536, help="serving: frames per launch")
    ap.add_argument("--serve-streams", type=int, default=4, help="serving: batches in flight")
    ap.add_argument("--serve-resume-step", type=int, default=0,
                    help="serving: TEP weights per window of a long frame (0: frames searched whole in their batch)")
    args = ap.parse_args()
    if args.membership == "solve" and not (args.config or "").startswith("c5"):
        ap.error("--membership solve applies to the serving configs (c5, c5long, c5adv); the decode "
                 "records report the solve path under their 'solve' key")
    if args.membership == "solve" and args.serve_resume_step:
        ap.error("--membership solve has no TEP search to continue (--serve-resume-step 0)")
    cfg = dict(CONFIGS[args.config or "c2"])
    cfg["name"] = args.config or "c2"
    if args.frames:
        cfg["frames"] = args.frames
    if args.impl == "reference":
        return run_reference(args, cfg)

    import torch

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl")
    import paper_2405_01808_gb300 as g

    if rank == 0:
        g.build()
    if dist:
        dist.barrier()
    g.lib()

    if cfg["kind"] == "bler":
        rows, fps = run_bler(args, cfg, g)
        if rank == 0:
            print(json.dumps({"metric": "BLER vs Eb/N0 (own curves; the paper's Fig. 4 values are not in its text)",
                              "value": fps, "unit": "frames/s (decode calls of the sweep)", "n_gpus": world,
                              "steps": len(rows), "warmup": 0, "higher_is_better": True, "dtype": "u32",
                              "data": "synthetic (seeded random polar codewords over AWGN)",
                              "config": {"workload": cfg["desc"], "frames_per_point": cfg["frames"]},
                              "bler": rows}), flush=True)
        return 0
    if cfg["kind"] in ("orders", "membership"):
        clocks = ClockSampler(local)
        clocks.start()
        rows = run_orders(args, cfg, g) if cfg["kind"] == "orders" else run_membership(args, cfg, g)
        clk = clocks.stop()
        if rank == 0:
            print(json.dumps({"metric": "TEP order comparison (queries, BLER)" if cfg["kind"] == "orders"
                              else "membership-test ablation (checks/s)",
                              "value": rows[0]["useful_checks_per_s"], "unit": "checks/s (first row)",
                              "n_gpus": world, "steps": 1, "warmup": 1, "higher_is_better": True, "dtype": "u32",
                              "data": "synthetic (seeded random polar codewords over AWGN)",
                              "config": {"workload": cfg["desc"]}, "clocks": clk, "rows": rows}), flush=True)
        return 0
    ctx = {"rank": rank, "world": world, "dist": dist, "local": local}
    if cfg["kind"] == "serve":
        line = run_serve_config(args, cfg, g, ctx)
        if rank == 0:
            print(json.dumps(line), flush=True)
        return 0

    line = run_config(args, cfg, g, ctx)
    if args.config is None and not args.no_subconfigs:
        # the other throughput workloads, each measured the same way, as
        # sub-records of the headline line
        subs = {}
        for name in [c for c in args.subconfigs.split(",") if c]:
            sub = dict(CONFIGS[name])
            sub["name"] = name
            gc.collect()
            torch.cuda.empty_cache()
            if sub["kind"] == "serve":  # one rate and fewer requests inside the default run
                if name == "c5":
                    sub.update(rates=(2e6,), frames=300000,
                               desc=sub["desc"].replace("0.5/1/2/5 M frames/s", "2 M frames/s").replace(
                                   "1000000 requests per rate", "300000 requests"))
                rec = run_serve_config(args, sub, g, ctx)
            else:
                rec = run_config(args, sub, g, ctx)
            if rec is not None:
                rec.pop("metric", None)
                rec.pop("n_gpus", None)
                subs[name] = rec
        if line is not None:
            line["configs"] = subs
    if rank == 0:
        print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
