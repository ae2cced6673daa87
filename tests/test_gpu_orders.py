"""GPU parity of the TEP order variants and the membership tests: the
nearer-axis-first order (split search and per-TEP kernel), the five-point NNE
order (per-TEP kernel), the syndrome-delta and row-parity tests kept for
comparison, and the hash-join decision, each against the CPU oracle with the
same order, bit-exact on decoded words, query counts and abandon flags."""
from __future__ import annotations

import os

import numpy as np
import pytest

import workloads as wl

pytestmark = pytest.mark.gpu

THREADS = max(1, (os.cpu_count() or 1))


@pytest.fixture(scope="module")
def g():
    import torch

    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2405_01808_gb300 as grand

    grand.build()
    return grand


_codes = {}


def code_pair(g, oracle_lib, N):
    if N not in _codes:
        _codes[N] = (g.Code.polar(N, N // 2), oracle_lib.parity_H(N, N // 2), oracle_lib.info_set(N, N // 2))
    return _codes[N]


def to_dev(a):
    import torch

    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def unpack(r):
    import torch

    torch.cuda.synchronize()
    return {"cw": r["cw"].cpu().numpy().view(np.uint32),
            "queries": r["queries"].cpu().numpy().view(np.uint32).astype(np.int64),
            "abandon": r["abandon"].cpu().numpy()}


def assert_same(got, want, label=""):
    bad = np.nonzero((got["queries"] != want["queries"]) | (got["abandon"] != want["abandon"]) |
                     (got["cw"] != want["cw"]).any(axis=1))[0]
    assert bad.size == 0, (f"{label}: {bad.size} frames differ, first {bad[:8].tolist()}: "
                           f"gpu q={got['queries'][bad[:4]].tolist()} ab={got['abandon'][bad[:4]].tolist()} "
                           f"oracle q={want['queries'][bad[:4]].tolist()} ab={want['abandon'][bad[:4]].tolist()}")


# oracle order ids: 1 paper, 2 nearer axis first, 3 five-point NNE (same as the ABI's)
NNE, NEARER, NNE5 = 1, 2, 3
AUTO, DELTA, ROW, HASH = 0, 1, 2, 3

CASES = [
    # order, membership, N, M, S, EbN0 dB, cap, frames, lik
    (NEARER, AUTO, 128, 16, 10, 7.0, 1 << 20, 200, 0),
    (NEARER, AUTO, 256, 64, 9, 10.0, 4 ** 9, 150, 0),
    (NEARER, AUTO, 32, 4, 8, 3.0, 1 << 16, 300, 0),
    (NEARER, AUTO, 128, 16, 10, 7.0, 1 << 20, 120, 1),
    (NEARER, DELTA, 128, 16, 8, 7.0, 1 << 16, 200, 0),
    (NEARER, ROW, 64, 16, 6, 6.0, 4 ** 6, 200, 0),
    (NNE, DELTA, 128, 16, 10, 6.0, 1 << 20, 100, 0),
    (NNE, DELTA, 32, 4, 8, 3.0, 1 << 16, 300, 0),
    (NNE, DELTA, 512, 64, 11, 13.0, 50000, 80, 0),
    (NNE, ROW, 128, 16, 8, 7.0, 1 << 16, 150, 0),
    (NNE, ROW, 1024, 256, 12, 17.0, 1 << 14, 30, 0),
    (NNE, ROW, 256, 4096, 10, 24.0, 1 << 16, 60, 1),
    (NNE5, AUTO, 128, 16, 8, 7.0, 5 ** 8, 160, 0),
    (NNE5, AUTO, 32, 4, 8, 3.0, 5 ** 8, 300, 0),
    (NNE5, AUTO, 256, 64, 10, 10.0, 1 << 20, 80, 0),
    (NNE5, AUTO, 128, 1024, 8, 20.0, 1 << 16, 100, 0),
    (NNE5, AUTO, 32, 4096, 8, 24.0, 1 << 16, 100, 0),   # L = 3 < S
    (NNE5, AUTO, 128, 16, 0, 8.0, 100, 60, 0),          # S = 0
    (NNE5, AUTO, 512, 64, 7, 12.0, 3000, 60, 0),        # cap inside a weight class
    (NNE5, ROW, 128, 16, 6, 6.0, 5 ** 6, 150, 0),
    (NNE, HASH, 128, 16, 10, 6.0, 1 << 20, 200, 0),
    (NNE, HASH, 128, 16, 10, 10.0, 1 << 20, 400, 0),
    (NNE, HASH, 32, 4, 8, 3.0, 1 << 16, 300, 0),
    (NNE, HASH, 256, 64, 9, 10.0, 4 ** 9, 150, 0),
    (NNE, HASH, 512, 64, 10, 13.0, 50000, 100, 0),      # cap inside a weight class
    (NNE, HASH, 1024, 256, 10, 17.0, 1 << 14, 40, 0),
    (NNE, HASH, 128, 16, 1, 8.0, 100, 200, 0),           # S = 1
    (NNE, HASH, 128, 16, 12, 9.0, 1 << 20, 60, 0),       # S' = 12: 6-rank sides
    (NNE, HASH, 512, 64, 12, 13.0, 1 << 22, 40, 0),
    (NNE, HASH, 1024, 256, 11, 17.0, 1 << 20, 30, 0),    # S' = 11: 5 + 6 ranks
    (NEARER, HASH, 128, 16, 10, 7.0, 1 << 20, 150, 0),
    (NNE, HASH, 128, 16, 10, 7.0, 1 << 20, 100, 1),      # literal likelihood
]


@pytest.mark.parametrize("order,mem,N,M,S,snr,cap,F,lik", CASES)
def test_order_parity(g, oracle_lib, order, mem, N, M, S, snr, cap, F, lik):
    code, H, info = code_pair(g, oracle_lib, N)
    d = wl.qam_frames(50 + order, N + M + S, F, N, info, M, snr)
    want = oracle_lib.decode_qam(H, d["symbols"], M, S, cap, literal=bool(lik), threads=THREADS, order=order)
    p = g.Params.make(order=order, M=M, S=S, query_cap=cap, lik_variant=lik, membership=mem)
    got = unpack(g.decode_symbols(code, p, to_dev(d["symbols"])))
    assert_same(got, want, f"order={order} membership={mem} N={N} M={M} S={S}")


@pytest.mark.parametrize("mem", [DELTA, ROW, HASH])
def test_membership_tests_equal_split_search(g, oracle_lib, mem):
    """The per-TEP kernel with either membership test decides exactly as the
    split search on a larger batch (the paper's order)."""
    N, M, S = 128, 16, 10
    code, H, info = code_pair(g, oracle_lib, N)
    d = wl.qam_frames(61, mem, 2000, N, info, M, 9.0)
    sym = to_dev(d["symbols"])
    a = unpack(g.decode_symbols(code, g.Params.make(M=M, S=S, query_cap=1 << 18), sym))
    b = unpack(g.decode_symbols(code, g.Params.make(M=M, S=S, query_cap=1 << 18, membership=mem), sym))
    assert_same(b, a, f"membership={mem}")


def test_nearer_two_call_path_and_mixed(g, oracle_lib):
    """The nearer order through grand_decode_batch (nmask bit 32 from
    grand_demod) and through an uneven batch equals the fused call and the
    oracle."""
    import torch

    N, M, S = 128, 16, 10
    code, H, info = code_pair(g, oracle_lib, N)
    d = wl.qam_frames(62, 0, 300, N, info, M, 7.0)
    sym = to_dev(d["symbols"])
    p = g.Params.make(order=NEARER, M=M, S=S, query_cap=1 << 20)
    dm = g.demod(sym, M, N)
    a = unpack(g.decode_batch(code, p, dm["y"], dm["hard_idx"], dm["key"], dm["nmask"]))
    b = unpack(g.decode_symbols(code, p, sym))
    assert_same(a, b, "two-call")
    want = oracle_lib.decode_qam(H, d["symbols"], M, S, 1 << 20, threads=THREADS, order=NEARER)
    assert_same(b, want, "fused vs oracle")
    L = wl.symbols_per_frame(N, M)
    F = d["symbols"].shape[0]
    desc = g.frame_desc(np.zeros(F, np.int64), np.full(F, M), np.arange(F) * L, np.arange(F) * (N // 32))
    r = g.decode_mixed([code], p, to_dev(desc.view(np.uint8)), sym.reshape(-1), F * (N // 32))
    torch.cuda.synchronize()
    mixed = {"cw": r["cw"].cpu().numpy().view(np.uint32).reshape(F, N // 32),
             "queries": r["queries"].cpu().numpy().view(np.uint32).astype(np.int64),
             "abandon": r["abandon"].cpu().numpy()}
    assert_same(mixed, want, "mixed vs oracle")


def test_per_tep_edge_cases(g, oracle_lib):
    """Non-finite frames, an empty batch and the statistics of the per-TEP
    kernel."""
    import torch

    N, M = 128, 16
    code, H, info = code_pair(g, oracle_lib, N)
    d = wl.qam_frames(63, 0, 50, N, info, M, 7.0)
    s = d["symbols"].copy()
    s[2, 3] = np.complex64(complex(np.nan, 0.0))
    s[40, 0] = np.complex64(complex(0.0, -np.inf))
    for order, mem in ((NNE5, AUTO), (NNE, ROW)):
        cap = 5 ** 7 if order == NNE5 else 4 ** 7
        want = oracle_lib.decode_qam(H, s, M, 7, cap, threads=THREADS, order=order)
        p = g.Params.make(order=order, M=M, S=7, query_cap=cap, membership=mem)
        r = g.decode_symbols(code, p, to_dev(s), stats=True)
        got = unpack(r)
        assert_same(got, want, f"order={order} membership={mem}")
        assert got["abandon"][2] == 2 and got["abandon"][40] == 2
        hard = (got["queries"] > 1) | (got["abandon"] == 1)
        assert r["hard_frames"] == int(hard.sum())
        assert r["evaluated_checks"] >= int(got["queries"][got["abandon"] != 2].sum())
        e = g.decode_symbols(code, p, torch.zeros((0, 32), dtype=torch.complex64, device="cuda"), stats=True)
        torch.cuda.synchronize()
        assert e["cw"].shape == (0, 4) and e["hard_frames"] == 0


def test_unsupported_combinations_are_refused(g, oracle_lib):
    import torch

    N, M = 128, 16
    code, _, _ = code_pair(g, oracle_lib, N)
    sym = torch.zeros((4, 32), dtype=torch.complex64, device="cuda")
    dm = g.demod(sym, M, N)
    with pytest.raises(g.GrandError):  # the hash join does not serve the five-point order
        g.decode_symbols(code, g.Params.make(order=NNE5, M=M, S=8, membership=HASH), sym)
    for p in (g.Params.make(order=NNE5, M=M, S=8), g.Params.make(M=M, S=8, membership=ROW)):
        with pytest.raises(g.GrandError):
            g.decode_batch(code, p, dm["y"], dm["hard_idx"], dm["key"], dm["nmask"])
        desc = g.frame_desc([0] * 4, [M] * 4, np.arange(4) * 32, np.arange(4) * 4)
        with pytest.raises(g.GrandError):
            g.decode_mixed([code], p, to_dev(desc.view(np.uint8)), sym.reshape(-1), 16)
    with pytest.raises(g.GrandError):  # S above the five-point limit
        g.decode_symbols(code, g.Params.make(order=NNE5, M=M, S=11), sym)
    with pytest.raises(g.GrandError):  # unknown membership test
        g.decode_symbols(code, g.Params.make(M=M, S=8, membership=4), sym)


def test_hash_join_two_call_mixed_and_full_batch(g, oracle_lib):
    """The hash join through grand_decode_batch and an uneven batch, and on a
    large batch against the split search (every output identical)."""
    import torch

    N, M, S = 128, 16, 10
    code, H, info = code_pair(g, oracle_lib, N)
    d = wl.qam_frames(64, 0, 30000, N, info, M, 7.0)
    sym = to_dev(d["symbols"])
    ph = g.Params.make(M=M, S=S, query_cap=1 << 20, membership=HASH)
    a = unpack(g.decode_symbols(code, g.Params.make(M=M, S=S, query_cap=1 << 20), sym))
    b = unpack(g.decode_symbols(code, ph, sym))
    assert_same(b, a, "hash vs split, 30000 frames")
    dm = g.demod(sym, M, N)
    c = unpack(g.decode_batch(code, ph, dm["y"], dm["hard_idx"], dm["key"], dm["nmask"]))
    assert_same(c, a, "hash two-call")
    Ns = (32, 64, 128, 256, 512, 1024)
    codes = [code_pair(g, oracle_lib, n)[0] for n in Ns]
    infos = {n: code_pair(g, oracle_lib, n)[2] for n in Ns}
    mx = wl.mixed_frames(65, 0, 3000, infos)
    desc = g.frame_desc(np.searchsorted(np.array(Ns), mx["N"]), mx["M"], mx["sym_offset"], mx["cw_offset"])
    dd, ss = to_dev(desc.view(np.uint8)), to_dev(mx["symbols"])
    pm = g.Params.make(M=0, S=10, query_cap=1 << 18)
    pmh = g.Params.make(M=0, S=10, query_cap=1 << 18, membership=HASH)
    r1 = g.decode_mixed(codes, pm, dd, ss, mx["n_cw_words"])
    r2 = g.decode_mixed(codes, pmh, dd, ss, mx["n_cw_words"])
    torch.cuda.synchronize()
    for k in ("cw", "queries", "abandon"):
        assert torch.equal(r1[k], r2[k]), k
