"""Parity at the full workload sizes, in the launch configuration the benchmark
times: each whole batch is decoded on the GPU and compared frame by frame with
the oracle's expected outputs stored under tests/golden/ (written offline by
tests/golden/make_fullsize_golden.py, which calls only the oracle and the input
generator). Decoded words, query counts and abandon flags must be identical
(Alg. 2 Step 5: the first valid TEP in canonical order with a zero syndrome;
abandonment at the query cap, Sec. II).

Coverage (the stored counts; each stratum is a prefix of its frames, so
abandoning frames appear in their natural share):
  * N=128 16-QAM, S=10, cap 2^20: every frame of the 300,000-frame batch.
  * N=512 64-QAM and N=1024 256-QAM, S=12, cap 2^24: per Eb/N0 point the
    first n frames of 20,000, n as stored (up to 2,000; fewer where the
    oracle's 2^24-query abandons exhaust the generator's host-time budget).
  * the uneven 1,000,000-frame mix (S=min(L,10), cap 2^20): per (N, M) class
    the first n frames of the class in batch order (up to 2,000).
Every other frame of each batch is checked for the properties that hold at
any size: a decoded word is a codeword (H x = 0), an abandoned frame returns
its hard word, queries never exceed the cap."""
from __future__ import annotations

import hashlib
import json
import os

import numpy as np
import pytest

import workloads as wl

pytestmark = pytest.mark.gpu

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")
UNIFORM = {
    "c2": dict(cid=2, N=128, M=16, snrs=(6.0, 8.0, 10.0), frames=100000, S=10, cap=1 << 20),
    "c3a": dict(cid=3, N=512, M=64, snrs=(10.0, 12.0, 14.0, 16.0), frames=20000, S=12, cap=1 << 24),
    "c3b": dict(cid=4, N=1024, M=256, snrs=(10.0, 12.0, 14.0, 16.0), frames=20000, S=12, cap=1 << 24),
}


@pytest.fixture(scope="module")
def g():
    import torch

    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2405_01808_gb300 as grand

    grand.build()
    return grand


def load_golden(config):
    path = os.path.join(GOLDEN, f"fullsize_{config}.npz")
    assert os.path.exists(path), f"missing {path}: run tests/golden/make_fullsize_golden.py --config {config}"
    z = np.load(path, allow_pickle=False)
    return z, json.loads(str(z["meta"]))


def sha(sym):
    return hashlib.sha256(np.ascontiguousarray(sym, dtype=np.complex64).tobytes()).hexdigest()


def compare_stratum(oracle_lib, z, name, st, sym, cw, q, ab):
    """Every stored frame of one stratum: (sym, cw, q, ab) are the stratum's
    frames in order, from its first frame."""
    n = int(st["n"])
    assert n > 0
    assert sha(sym[:n]) == st["symbols_sha256"], f"{name}: the input generator no longer reproduces the stored batch"
    y = oracle_lib.demod(sym[:n], st["M"], st["N"])["y"]
    want_cw = y ^ z[f"{name}_e"]
    want_q = z[f"{name}_queries"].astype(np.int64)
    want_ab = z[f"{name}_abandon"]
    bad_q = np.nonzero(want_q != q[:n])[0]
    bad_ab = np.nonzero(want_ab != ab[:n])[0]
    bad_cw = np.nonzero((want_cw != cw[:n]).any(axis=1))[0]
    assert bad_q.size == 0 and bad_ab.size == 0 and bad_cw.size == 0, (
        f"{name}: {bad_q.size} query counts, {bad_ab.size} abandon flags, {bad_cw.size} words differ "
        f"(first frames {bad_q[:5].tolist()} {bad_ab[:5].tolist()} {bad_cw[:5].tolist()})")
    return n, int((want_ab == 1).sum())


def check_properties(H_dense, cw, queries, abandon, y, cap):
    """Decoded words satisfy H x = 0; abandoned frames return y; queries <= cap."""
    N = H_dense.shape[1]
    bits = ((cw[:, :, None] >> np.arange(32, dtype=np.uint32)) & 1).reshape(len(cw), N).astype(np.uint8)
    dec = abandon == 0
    # float32 products are exact here (sums of at most N ones)
    syn = np.rint(bits[dec].astype(np.float32) @ H_dense.T.astype(np.float32)).astype(np.int64) % 2
    assert not syn.any(), "a decoded word is not a codeword"
    assert np.array_equal(cw[abandon == 1], y[abandon == 1]), "an abandoned frame does not return its hard word"
    assert np.all(queries <= cap) and np.all(queries >= 1)
    assert set(np.unique(abandon).tolist()) <= {0, 1}


@pytest.mark.parametrize("config", ["c2", "c3a", "c3b"])
def test_uniform_full_batch(g, oracle_lib, config):
    """The whole batch (every SNR point) in one fused call, as the benchmark
    times it; every stored frame equal to the oracle's."""
    import torch

    c = UNIFORM[config]
    z, meta = load_golden(config)
    N, K, M = c["N"], c["N"] // 2, c["M"]
    info = oracle_lib.info_set(N, K)
    parts = [wl.qam_frames(c["cid"], i, c["frames"], N, info, M, snr) for i, snr in enumerate(c["snrs"])]
    sym = np.concatenate([p["symbols"] for p in parts])
    code = g.Code.polar(N, K)
    try:
        p = g.Params.make(M=M, S=c["S"], query_cap=c["cap"])
        r = g.decode_symbols(code, p, torch.from_numpy(sym).cuda())
        torch.cuda.synchronize()
        cw = r["cw"].cpu().numpy().view(np.uint32)
        q = r["queries"].cpu().numpy().view(np.uint32).astype(np.int64)
        ab = r["abandon"].cpu().numpy()
    finally:
        code.close()
    H = oracle_lib.parity_H(N, K)
    check_properties(H, cw, q, ab, oracle_lib.demod(sym, M, N)["y"], c["cap"])
    compared = 0
    for i in range(len(c["snrs"])):
        name = f"s{i}"
        assert name in meta["strata"], f"{config}: stratum {name} missing from the stored outputs"
        st = meta["strata"][name]
        lo = i * c["frames"]
        n, _ = compare_stratum(oracle_lib, z, name, st, sym[lo:lo + c["frames"]], cw[lo:lo + c["frames"]],
                               q[lo:lo + c["frames"]], ab[lo:lo + c["frames"]])
        compared += n
    if config == "c2":
        assert compared == len(sym), "every frame of the N=128 batch is compared"


def test_uneven_mix_full_batch(g, oracle_lib):
    """1,000,000 mixed frames through the autotuned CUDA-graph plan, as timed;
    every stored frame of every (N, M) class equal to the oracle's."""
    import torch

    z, meta = load_golden("c4")
    Ns = wl.MIXED_N
    codes = [g.Code.polar(n, n // 2) for n in Ns]
    info = {n: oracle_lib.info_set(n, n // 2) for n in Ns}
    mx = wl.mixed_frames(5, 1000, 1000000, info)
    desc = torch.from_numpy(g.frame_desc(np.searchsorted(np.array(Ns), mx["N"]), mx["M"], mx["sym_offset"],
                                         mx["cw_offset"]).view(np.uint8)).cuda()
    sym = torch.from_numpy(mx["symbols"]).cuda()
    p = g.Params.make(M=0, S=10, query_cap=1 << 20)
    g.autotune_mixed(codes, p, desc[: 100000 * g.FRAME_DESC_DTYPE.itemsize], sym, mx["n_cw_words"])
    cw_d = torch.empty(mx["n_cw_words"], dtype=torch.int32, device="cuda")
    q_d = torch.empty(1000000, dtype=torch.int32, device="cuda")
    ab_d = torch.empty(1000000, dtype=torch.uint8, device="cuda")
    plan = g.plan_mixed(codes, p, desc, sym, cw_d, q_d, ab_d)
    plan.launch()
    torch.cuda.synchronize()
    cw = cw_d.cpu().numpy().view(np.uint32)
    q = q_d.cpu().numpy().view(np.uint32).astype(np.int64)
    ab = ab_d.cpu().numpy()
    plan.close()
    for c in codes:
        c.close()
    classes = 0
    for n in Ns:
        H = oracle_lib.parity_H(n, n // 2)
        for M in wl.QAM_ORDERS:
            f = np.nonzero((mx["N"] == n) & (mx["M"] == M))[0]
            L = wl.symbols_per_frame(n, M)
            symf = mx["symbols"][mx["sym_offset"][f][:, None] + np.arange(L)[None, :]]
            cwf = cw[mx["cw_offset"][f][:, None] + np.arange(n // 32)[None, :]]
            y = oracle_lib.demod(symf, M, n)["y"]
            check_properties(H, cwf, q[f], ab[f], y, 1 << 20)
            name = f"n{n}_m{M}"
            assert name in meta["strata"], f"c4: class {name} missing from the stored outputs"
            compare_stratum(oracle_lib, z, name, meta["strata"][name], symf, cwf, q[f], ab[f])
            classes += 1
    assert classes == len(Ns) * len(wl.QAM_ORDERS)
