#!/usr/bin/env python3
"""Write the oracle's expected outputs for the full-size workloads.

This script calls only the CPU oracle (`oracle/`) and the seeded input
generator (`workloads/`); nothing here comes from the CUDA library. It
regenerates the batches the benchmark times and decodes them frame by frame
with the oracle's plain sequential GRAND (Alg. 2 Step 5: valid TEPs in
canonical order, a dense H (y xor e) per query, stop at the first codeword or
at the query cap; abandonment as in Sec. II):

  c2   polar N=128 K=64, 16-QAM, Eb/N0 6/8/10 dB x 100,000 frames, S=10,
       cap 2^20 -- every frame
  c3a  polar N=512 K=256, 64-QAM, Eb/N0 10/12/14/16 dB x 20,000, S=12, cap 2^24
  c3b  polar N=1024 K=512, 256-QAM, the same SNR points, S=12, cap 2^24
  c4   the uneven mix (N 32..1024 x M 4..256, Eb/N0 U(4,14) dB), 1,000,000
       frames, S=min(L,10), cap 2^20

For c3a/c3b each SNR point is a stratum and for c4 each (N, M) class is one.
A stratum's expected outputs cover a PREFIX of its frames (frames 0..n-1 of
the SNR batch; for c4 the first n frames of the class in batch order), so
abandoning frames are kept in their natural share. n is at most --max-frames
and stops earlier when the stratum's --budget-s of host time is spent (a
2^24-query abandon costs the oracle 15-25 s of one core); the stored count
says how far it got. Work is resumable: a stratum already in the output file
with n frames continues from frame n.

Stored per stratum (numpy .npz, compressed): queries (uint32), abandon (uint8),
e = cw xor y (uint32 words; y = the oracle's hard word, so e is the decoded
error pattern and mostly zero), and the SHA-256 of the stratum's received
symbols, so a test can tell a changed input generator from a decoding
mismatch.

  python tests/golden/make_fullsize_golden.py --config c2 --threads 6
"""
from __future__ import annotations

import argparse
import concurrent.futures as cf
import hashlib
import json
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import oracle  # noqa: E402
import workloads as wl  # noqa: E402

# The benchmark's batches: config id of the seed, SNR points (one seed stream
# each, stream = SNR index), frames per point.
UNIFORM = {
    "c2": dict(cid=2, N=128, M=16, snrs=(6.0, 8.0, 10.0), frames=100000, S=10, cap=1 << 20),
    "c3a": dict(cid=3, N=512, M=64, snrs=(10.0, 12.0, 14.0, 16.0), frames=20000, S=12, cap=1 << 24),
    "c3b": dict(cid=4, N=1024, M=256, snrs=(10.0, 12.0, 14.0, 16.0), frames=20000, S=12, cap=1 << 24),
}
MIXED = dict(cid=5, stream=1000, frames=1000000, S=10, cap=1 << 20)


def out_path(config: str) -> str:
    return os.path.join(HERE, f"fullsize_{config}.npz")


def symbols_sha(sym: np.ndarray) -> str:
    return hashlib.sha256(np.ascontiguousarray(sym, dtype=np.complex64).tobytes()).hexdigest()


def load(config: str) -> dict:
    p = out_path(config)
    if not os.path.exists(p):
        return {}
    with np.load(p, allow_pickle=False) as z:
        return {k: z[k] for k in z.files}


def save(config: str, arrays: dict, meta: dict) -> None:
    p = out_path(config)
    tmp = p + ".tmp.npz"
    np.savez_compressed(tmp, meta=np.array(json.dumps(meta, sort_keys=True)), **arrays)
    os.replace(tmp, p)


def strata(config: str):
    """(name, symbols (n_all, L), N, M, S, cap, description) per stratum."""
    if config in UNIFORM:
        c = UNIFORM[config]
        info = oracle.info_set(c["N"], c["N"] // 2)
        for i, snr in enumerate(c["snrs"]):
            d = wl.qam_frames(c["cid"], i, c["frames"], c["N"], info, c["M"], snr)
            yield (f"s{i}", d["symbols"], c["N"], c["M"], c["S"], c["cap"],
                   dict(ebn0_db=snr, stream=i, first_frame=i * c["frames"]))
        return
    info = {n: oracle.info_set(n, n // 2) for n in wl.MIXED_N}
    mx = wl.mixed_frames(MIXED["cid"], MIXED["stream"], MIXED["frames"], info)
    for n in wl.MIXED_N:
        for M in wl.QAM_ORDERS:
            f = np.nonzero((mx["N"] == n) & (mx["M"] == M))[0]
            L = wl.symbols_per_frame(n, M)
            sym = mx["symbols"][mx["sym_offset"][f][:, None] + np.arange(L)[None, :]]
            yield (f"n{n}_m{M}", sym, n, M, min(MIXED["S"], L), MIXED["cap"],
                   dict(class_frames=int(f.size), note="first n frames of the class in batch order"))


def run_stratum(H, sym, M, S, cap, start, stop_at, deadline, threads, chunk):
    """Decode frames start..stop_at-1 in order on a thread pool (the oracle call
    releases the GIL); stop submitting at `deadline` (time.time()). Every
    submitted chunk is waited for, so the outputs form a prefix. Returns
    (end of the prefix, outputs or None)."""
    results = []
    nxt = start
    with cf.ThreadPoolExecutor(max_workers=threads) as ex:
        pending = []
        while nxt < stop_at and time.time() < deadline:
            while len(pending) < 2 * threads and nxt < stop_at and time.time() < deadline:
                hi = min(nxt + chunk, stop_at)
                pending.append((nxt, ex.submit(oracle.decode_qam, H, sym[nxt:hi], M, S, cap, threads=1)))
                nxt = hi
            cf.wait([f for _, f in pending], return_when=cf.FIRST_COMPLETED)
            while pending and pending[0][1].done():
                results.append(pending.pop(0)[1].result())
        for _, f in pending:
            results.append(f.result())
    if not results:
        return start, None
    return nxt, {k: np.concatenate([r[k] for r in results]) for k in ("queries", "abandon", "cw")}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--config", required=True, choices=["c2", "c3a", "c3b", "c4"])
    ap.add_argument("--threads", type=int, default=os.cpu_count() or 1)
    ap.add_argument("--max-frames", type=int, default=None,
                    help="frames per stratum (default: all for c2, 2000 otherwise)")
    ap.add_argument("--budget-s", type=float, default=float("inf"), help="host seconds per stratum and invocation")
    ap.add_argument("--chunk", type=int, default=None, help="frames per oracle call")
    ap.add_argument("--segment", type=int, default=10000, help="frames between saves")
    ap.add_argument("--only", default=None, help="comma-separated stratum names to work on")
    args = ap.parse_args()
    max_frames = args.max_frames if args.max_frames is not None else (
        UNIFORM["c2"]["frames"] if args.config == "c2" else 2000)
    chunk = args.chunk or (50 if args.config == "c2" else (1 if args.config.startswith("c3") else 8))
    have = load(args.config)
    meta = json.loads(str(have["meta"])) if "meta" in have else {}
    meta.setdefault("strata", {})
    meta["config"] = args.config
    meta["generator"] = "tests/golden/make_fullsize_golden.py (oracle + workloads only)"
    with open(os.path.join(ROOT, "oracle", "grand_oracle.c"), "rb") as fh:
        meta["oracle_c_sha256"] = hashlib.sha256(fh.read()).hexdigest()
    arrays = {k: v for k, v in have.items() if k != "meta"}
    only = set(args.only.split(",")) if args.only else None
    for name, sym, N, M, S, cap, desc in strata(args.config):
        if only is not None and name not in only:
            continue
        n_all = len(sym)
        target = min(max_frames, n_all)
        n_have = int(meta["strata"].get(name, {}).get("n", 0))
        if n_have >= target:
            print(f"{args.config}/{name}: {n_have} frames already", flush=True)
            continue
        H = oracle.parity_H(N, N // 2)
        t0 = time.time()
        deadline = t0 + args.budget_s
        while n_have < target and time.time() < deadline:
            seg_stop = min(n_have + args.segment, target)
            pos, r = run_stratum(H, sym, M, S, cap, n_have, seg_stop, deadline, args.threads, chunk)
            if r is None:
                break
            y = oracle.demod(sym[n_have:pos], M, N)["y"]
            e = (r["cw"] ^ y).astype(np.uint32)
            q = r["queries"].astype(np.uint32)
            ab = r["abandon"].astype(np.uint8)
            if n_have:
                e = np.concatenate([arrays[f"{name}_e"], e])
                q = np.concatenate([arrays[f"{name}_queries"], q])
                ab = np.concatenate([arrays[f"{name}_abandon"], ab])
            arrays[f"{name}_e"], arrays[f"{name}_queries"], arrays[f"{name}_abandon"] = e, q, ab
            meta["strata"][name] = dict(desc, N=N, K=N // 2, M=M, S=S, cap=cap, n=int(pos), frames_in_batch=n_all,
                                        symbols_sha256=symbols_sha(sym[:pos]), abandons=int((ab == 1).sum()),
                                        useful_checks=int(q.astype(np.int64).sum()))
            save(args.config, arrays, meta)
            print(f"{args.config}/{name}: {n_have} -> {pos} of {n_all} frames, abandons {int((ab == 1).sum())}, "
                  f"{time.time() - t0:.0f} s", flush=True)
            n_have = pos

if __name__ == "__main__":
    main()
