"""Parity at the full workload sizes, in the launch configuration the benchmark
times: the whole batch is decoded on the GPU; a stratified sample of frames
(decoded at several query positions, abandoned, every code/constellation class)
is compared bit-exactly with the oracle, and every frame is checked for the
properties that hold at any size: a decoded word is a codeword (H x = 0), an
abandoned frame returns its hard word, queries never exceed the cap."""
from __future__ import annotations

import os

import numpy as np
import pytest

import workloads as wl

pytestmark = pytest.mark.gpu

THREADS = max(1, os.cpu_count() or 1)


@pytest.fixture(scope="module")
def g():
    import torch

    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2405_01808_gb300 as grand

    grand.build()
    return grand


def stratified(queries, abandon, per=12, seed=0):
    """Frame indices: decoded ones spread over the query-count range, plus abandons."""
    rng = np.random.default_rng(seed)
    dec = np.nonzero(abandon == 0)[0]
    ab = np.nonzero(abandon == 1)[0]
    out = []
    if dec.size:
        order = dec[np.argsort(queries[dec], kind="stable")]
        out += order[np.linspace(0, order.size - 1, min(per, order.size)).astype(int)].tolist()
    if ab.size:
        out += rng.choice(ab, size=min(per // 3, ab.size), replace=False).tolist()
    return np.unique(np.array(out, dtype=np.int64))


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


def test_n128_16qam_full_batch(g, oracle_lib):
    """300,000 frames (Eb/N0 6/8/10 dB x 100,000), S=10, cap 2^20, one fused call."""
    import torch

    N, K, M, S, cap = 128, 64, 16, 10, 1 << 20
    code = g.Code.polar(N, K)
    _, frozen = g.polar_H(N, K)
    info = np.setdiff1d(np.arange(N), frozen)
    parts = [wl.qam_frames(2, i, 100000, N, info, M, snr) for i, snr in enumerate((6.0, 8.0, 10.0))]
    sym = np.concatenate([p["symbols"] for p in parts])
    p = g.Params.make(M=M, S=S, query_cap=cap)
    r = g.decode_symbols(code, p, torch.from_numpy(sym).cuda())
    torch.cuda.synchronize()
    cw = r["cw"].cpu().numpy().view(np.uint32)
    q = r["queries"].cpu().numpy().view(np.uint32).astype(np.int64)
    ab = r["abandon"].cpu().numpy()
    H = oracle_lib.parity_H(N, K)
    y = oracle_lib.demod(sym, M, N)["y"]
    check_properties(H, cw, q, ab, y, cap)
    for s in range(3):
        lo = s * 100000
        idx = lo + stratified(q[lo:lo + 100000], ab[lo:lo + 100000], per=18, seed=s)
        want = oracle_lib.decode_qam(H, sym[idx], M, S, cap, threads=THREADS)
        assert np.array_equal(want["queries"], q[idx]) and np.array_equal(want["abandon"], ab[idx])
        assert np.array_equal(want["cw"], cw[idx])


@pytest.mark.parametrize("N,M,snr", [(512, 64, 14.0), (1024, 256, 16.0)])
def test_s12_full_batch(g, oracle_lib, N, M, snr):
    """20,000 frames at one SNR point of the S=12, cap 2^24 workloads."""
    import torch

    K, S, cap = N // 2, 12, 1 << 24
    code = g.Code.polar(N, K)
    _, frozen = g.polar_H(N, K)
    info = np.setdiff1d(np.arange(N), frozen)
    d = wl.qam_frames(3 if N == 512 else 4, 7, 20000, N, info, M, snr)
    p = g.Params.make(M=M, S=S, query_cap=cap)
    r = g.decode_symbols(code, p, torch.from_numpy(d["symbols"]).cuda())
    torch.cuda.synchronize()
    cw = r["cw"].cpu().numpy().view(np.uint32)
    q = r["queries"].cpu().numpy().view(np.uint32).astype(np.int64)
    ab = r["abandon"].cpu().numpy()
    H = oracle_lib.parity_H(N, K)
    y = oracle_lib.demod(d["symbols"], M, N)["y"]
    check_properties(H, cw, q, ab, y, cap)
    idx = stratified(q, ab, per=15, seed=N)
    idx = idx[np.argsort(ab[idx])][:20]  # keep the oracle's share of 2^24-query abandons bounded
    want = oracle_lib.decode_qam(H, d["symbols"][idx], M, S, cap, threads=THREADS)
    assert np.array_equal(want["queries"], q[idx]) and np.array_equal(want["abandon"], ab[idx])
    assert np.array_equal(want["cw"], cw[idx])


def test_uneven_mix_full_batch(g, oracle_lib):
    """1,000,000 mixed frames through the autotuned CUDA-graph plan, as timed."""
    import torch

    Ns = wl.MIXED_N
    codes = [g.Code.polar(n, n // 2) for n in Ns]
    info = {}
    for n in Ns:
        _, frozen = g.polar_H(n, n // 2)
        info[n] = np.setdiff1d(np.arange(n), frozen)
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
    for n in Ns:
        H = oracle_lib.parity_H(n, n // 2)
        for M in wl.QAM_ORDERS:
            f = np.nonzero((mx["N"] == n) & (mx["M"] == M))[0]
            L = wl.symbols_per_frame(n, M)
            symf = mx["symbols"][mx["sym_offset"][f][:, None] + np.arange(L)[None, :]]
            cwf = cw[mx["cw_offset"][f][:, None] + np.arange(n // 32)[None, :]]
            y = oracle_lib.demod(symf, M, n)["y"]
            check_properties(H, cwf, q[f], ab[f], y, 1 << 20)
            pick = stratified(q[f], ab[f], per=4, seed=n + M)
            if n == 1024:
                pick = pick[np.argsort(ab[f][pick])][:4]
            want = oracle_lib.decode_qam(H, symf[pick], M, min(10, L), 1 << 20, threads=THREADS)
            assert np.array_equal(want["queries"], q[f][pick]), (n, M)
            assert np.array_equal(want["abandon"], ab[f][pick]), (n, M)
            assert np.array_equal(want["cw"], cwf[pick]), (n, M)
