"""GPU parity: the CUDA path (through the C ABI) against the CPU oracle on the
same seeded inputs. Integer outputs (hard points, keys, neighbour masks, hard
words, decoded words, query counts, abandon flags) must be bit-exact; the FP32
likelihood must be within 1e-5 relative (floor 1) of the FP64 oracle."""
from __future__ import annotations

import math
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


def code_pair(g, oracle_lib, N, K=None):
    K = N // 2 if K is None else K
    key = (N, K)
    if key not in _codes:
        _codes[key] = (g.Code.polar(N, K), oracle_lib.parity_H(N, K), oracle_lib.info_set(N, K))
    return _codes[key]


def to_dev(a):
    import torch

    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def u32(t):
    return t.cpu().numpy().view(np.uint32)


def gpu_decode(g, code, symbols, M, S, cap, lik=0, tiles=(0, 0, 0, 0), stats=False):
    import torch

    p = g.Params.make(order=g.ORDER_QAM_NNE, M=M, S=S, query_cap=cap, lik_variant=lik, tiles=tiles)
    r = g.decode_symbols(code, p, to_dev(symbols), N0=1.0, stats=stats)
    torch.cuda.synchronize()
    out = {"cw": u32(r["cw"]), "queries": u32(r["queries"]).astype(np.int64),
           "abandon": r["abandon"].cpu().numpy()}
    if stats:
        out["evaluated_checks"] = r["evaluated_checks"]
        out["hard_frames"] = r["hard_frames"]
    return out


def assert_same(got, want, label=""):
    bad = np.nonzero((got["queries"] != want["queries"]) | (got["abandon"] != want["abandon"]) |
                     (got["cw"] != want["cw"]).any(axis=1))[0]
    assert bad.size == 0, (f"{label}: {bad.size} frames differ, first {bad[:8].tolist()}: "
                           f"gpu q={got['queries'][bad[:4]].tolist()} ab={got['abandon'][bad[:4]].tolist()} "
                           f"oracle q={want['queries'][bad[:4]].tolist()} ab={want['abandon'][bad[:4]].tolist()}")


# ---------------------------------------------------------------------------
# demodulation
# ---------------------------------------------------------------------------

def adversarial_symbols(M, F, L, seed):
    """Uniform over a box around the constellation plus exact thresholds,
    exact points, far outliers and a few non-finite values."""
    side = int(math.isqrt(M))
    d = math.sqrt(3 * (math.log2(M) / 2) / (M - 1))
    rng = np.random.default_rng(seed)
    re = rng.uniform(-side - 2, side + 2, size=(F, L))
    im = rng.uniform(-side - 2, side + 2, size=(F, L))
    n = F * L
    flat_re, flat_im = re.reshape(-1), im.reshape(-1)
    k = n // 8
    flat_re[:k] = 2 * rng.integers(-side // 2, side // 2 + 1, size=k)          # thresholds
    flat_im[k:2 * k] = 2 * rng.integers(-side // 2, side // 2, size=k) + 1     # exact points
    flat_re[2 * k:2 * k + 16] = 1e6 * rng.choice([-1, 1], size=16)              # far outliers
    s = (re * d + 1j * im * d).astype(np.complex64)
    s.reshape(-1)[3 * k] = np.complex64(complex(np.nan, 0.0))
    s.reshape(-1)[3 * k + 5] = np.complex64(complex(0.0, np.inf))
    return s


@pytest.mark.parametrize("M", [4, 16, 64, 256, 1024, 4096])
@pytest.mark.parametrize("lik", [0, 1])
def test_demod_parity(g, oracle_lib, M, lik):
    import torch

    N = 512 if M != 4 else 256
    L = wl.symbols_per_frame(N, M)
    s = adversarial_symbols(M, 97, L, 10 * M + lik)  # ragged frame count
    o = oracle_lib.demod(s, M, N, literal=bool(lik))
    r = g.demod(to_dev(s), M, N, N0=0.5, lik_variant=lik)
    torch.cuda.synchronize()
    assert np.array_equal(r["hard_idx"].cpu().numpy().view(np.uint16), o["hard_idx"])
    assert np.array_equal(u32(r["key"]), o["key"])
    assert np.array_equal(r["nmask"].cpu().numpy(), o["nmask"])
    assert np.array_equal(u32(r["y"]), o["y"])
    rel = r["rel"].cpu().numpy().astype(np.float64)
    err = np.abs(rel - o["rel"]) / np.maximum(1.0, np.abs(o["rel"]))
    assert err.max() <= 1e-5


@pytest.mark.parametrize("lik", [0, 1])
def test_demod_hand_vectors(g, lik):
    """The hand-worked vectors of Def. III.1 / III.2 (tests/golden, derived on
    paper, independent of the oracle) through the device demodulator: hard
    point, key, neighbour mask and likelihood of the frame's first symbol."""
    import torch

    from tests.test_oracle_pins import _read_hand_vectors

    for t in _read_hand_vectors():
        M, rI, rQ = int(t[0]), float(t[1]), float(t[2])
        key = int(t[14]) if lik else int(t[8])
        Lx = float(t[15]) if lik else float(t[7])
        nmask = int(t[9]) | 32 * int(t[17] if lik else t[16])
        d = math.sqrt(3 * (math.log2(M) / 2) / (M - 1))
        N = 32
        frame = np.full((1, wl.symbols_per_frame(N, M)), complex(rI * d, rQ * d), dtype=np.complex64)
        r = g.demod(to_dev(frame), M, N, N0=1.0, lik_variant=lik)
        torch.cuda.synchronize()
        assert int(r["hard_idx"].cpu().numpy().view(np.uint16)[0, 0]) == int(t[10]), t
        assert int(u32(r["key"])[0, 0]) == key, t
        assert int(r["nmask"].cpu().numpy()[0, 0]) == nmask, t
        rel = float(r["rel"].cpu().numpy()[0, 0])
        assert abs(rel - Lx) <= 1e-5 * max(1.0, abs(Lx)), t


@pytest.mark.parametrize("M", [64, 4096])
def test_demod_unaligned_symbols(g, oracle_lib, M):
    """Symbols starting 8 bytes past a 16-byte boundary take the one-symbol-
    per-thread path; outputs equal the oracle's, as on the paired path."""
    import torch

    N = 512
    L = wl.symbols_per_frame(N, M)
    s = adversarial_symbols(M, 31, L, 7 * M)
    flat = torch.zeros(s.size + 1, dtype=torch.complex64, device="cuda")
    flat[1:] = torch.from_numpy(s.reshape(-1)).cuda()
    x = flat[1:].view(31, L)
    assert x.data_ptr() % 16 == 8
    o = oracle_lib.demod(s, M, N)
    r = g.demod(x, M, N)
    torch.cuda.synchronize()
    assert np.array_equal(r["hard_idx"].cpu().numpy().view(np.uint16), o["hard_idx"])
    assert np.array_equal(u32(r["key"]), o["key"])
    assert np.array_equal(r["nmask"].cpu().numpy(), o["nmask"])
    assert np.array_equal(u32(r["y"]), o["y"])


def test_demod_bpsk(g):
    import torch

    rng = np.random.default_rng(1)
    r = rng.standard_normal((33, 64)).astype(np.float32)
    r[0, 0] = -0.0
    r[1, 3] = np.nan
    out = g.demod(to_dev(r), 2, 64, N0=1.0)
    torch.cuda.synchronize()
    want = wl.pack_bits((np.nan_to_num(r, nan=0.0) < 0).astype(np.uint8))
    assert np.array_equal(u32(out["y"]), want)
    nm = out["nmask"].cpu().numpy()
    assert nm[1, 3] == 128 and nm.sum() == 128


def test_demod_rejects_bad_arguments(g):
    import ctypes

    import torch

    s = torch.zeros((2, 32), dtype=torch.complex64, device="cuda")
    with pytest.raises(g.GrandError):
        g.demod(s, 16, 128, N0=0.0)
    with pytest.raises(g.GrandArgumentError):  # the binding's own checks
        g.demod(s, 8, 128)
    with pytest.raises(g.GrandArgumentError):
        g.demod(s, 64, 128)  # L must be ceil(128/6) = 22
    # the library's checks, called directly (as a C caller would)
    y = torch.zeros((2, 4), dtype=torch.int32, device="cuda")
    P = lambda t: ctypes.c_void_p(t.data_ptr())
    L = g.lib()
    assert L.grand_demod(P(s), 2, 32, 8, 1.0, 0, None, None, None, None, P(y), 128, None) == -1  # M = 8
    assert L.grand_demod(P(s), 2, 32, 64, 1.0, 0, None, None, None, None, P(y), 128, None) == -1  # L != 22
    assert L.grand_demod(P(s), 2, 32, 16, float("nan"), 0, None, None, None, None, P(y), 128, None) == -1
    assert L.grand_demod(P(s), 2, 32, 16, 1.0, 2, None, None, None, None, P(y), 128, None) == -1  # lik variant


# ---------------------------------------------------------------------------
# symbol-level decoding
# ---------------------------------------------------------------------------

CASES = [
    # N, M, S, EbN0 dB, cap, frames, lik
    (128, 16, 10, 6.0, 1 << 20, 160, 0),     # 16-QAM, paper-size cut-off, mostly abandoning
    (128, 16, 10, 10.0, 1 << 20, 700, 0),    # mostly light hits
    (128, 16, 8, 8.0, 1 << 16, 300, 0),      # the paper's S = 8
    (32, 4, 8, 3.0, 1 << 16, 400, 0),        # QPSK, L = 16
    (32, 256, 8, 12.0, 1 << 16, 300, 0),     # L = 4 < S: S' = L
    (64, 16, 7, 6.0, 4 ** 7, 300, 0),
    (256, 64, 9, 10.0, 4 ** 9, 200, 0),      # 64-QAM with padding bits
    (512, 64, 11, 13.0, 50000, 120, 0),      # cap inside a weight class
    (128, 16, 10, 7.0, 1 << 20, 160, 1),     # literal likelihood variant
    (128, 16, 1, 8.0, 100, 300, 0),          # S = 1
    (128, 16, 0, 8.0, 100, 100, 0),          # S = 0: only the hard word
    (1024, 256, 12, 17.0, 1 << 14, 60, 0),   # largest code, cap binds early
    (128, 1024, 8, 20.0, 1 << 16, 200, 0),   # 1024-QAM, L = 13
    (256, 4096, 10, 24.0, 1 << 20, 120, 0),  # 4096-QAM, L = 22 (4 padding bits)
    (32, 4096, 8, 24.0, 1 << 16, 200, 0),    # L = 3 < S
]


@pytest.mark.parametrize("N,M,S,snr,cap,F,lik", CASES)
def test_decode_parity(g, oracle_lib, N, M, S, snr, cap, F, lik):
    code, H, info = code_pair(g, oracle_lib, N)
    d = wl.qam_frames(20 + N, int(snr * 10) + S, F, N, info, M, snr)
    want = oracle_lib.decode_qam(H, d["symbols"], M, S, cap, literal=bool(lik), threads=THREADS)
    got = gpu_decode(g, code, d["symbols"], M, S, cap, lik)
    assert_same(got, want, f"N={N} M={M} S={S}")


def test_two_call_path_equals_fused(g, oracle_lib):
    import torch

    N, M, S = 128, 16, 10
    code, H, info = code_pair(g, oracle_lib, N)
    d = wl.qam_frames(31, 0, 500, N, info, M, 7.0)
    sym = to_dev(d["symbols"])
    dm = g.demod(sym, M, N)
    p = g.Params.make(M=M, S=S, query_cap=1 << 20)
    a = g.decode_batch(code, p, dm["y"], dm["hard_idx"], dm["key"], dm["nmask"])
    b = g.decode_symbols(code, p, sym)
    torch.cuda.synchronize()
    for k in ("cw", "queries", "abandon"):
        assert torch.equal(a[k], b[k]), k


@pytest.mark.parametrize("tiles", [(1, 0, 0, 0), (4, 3, 1, 0), (8, 5, 3, 0), (2, 6, 2, 0), (8, 1, 0, 0)])
def test_tiles_do_not_change_results(g, oracle_lib, tiles):
    N, M, S = 128, 16, 10
    code, H, info = code_pair(g, oracle_lib, N)
    d = wl.qam_frames(32, 0, 300, N, info, M, 7.0)
    base = gpu_decode(g, code, d["symbols"], M, S, 1 << 20)
    other = gpu_decode(g, code, d["symbols"], M, S, 1 << 20, tiles=tiles)
    assert_same(other, base, f"tiles={tiles}")


@pytest.mark.parametrize("tiles", [(4, 6, 2, 0), (1, 0, 3, 6), (4, 0, 2, 8), (8, 5, 2, 0), (8, 0, 2, 0)])
def test_tiles_do_not_change_results_s12(g, oracle_lib, tiles):
    """S' = 12: the warp-per-frame search (5 + 7 ranks, automatic split, any
    warps per CTA and register budget) and the CTA search (explicit split)
    decide identically."""
    N, M, S = 512, 64, 12
    code, H, info = code_pair(g, oracle_lib, N)
    d = wl.qam_frames(35, 0, 200, N, info, M, 12.0)
    base = gpu_decode(g, code, d["symbols"], M, S, 1 << 22)
    other = gpu_decode(g, code, d["symbols"], M, S, 1 << 22, tiles=tiles)
    assert_same(other, base, f"tiles={tiles}")
    want = oracle_lib.decode_qam(H, d["symbols"][:40], M, S, 1 << 22, threads=THREADS)
    assert_same({k: v[:40] for k, v in base.items()}, want, "S=12 vs oracle")


def test_empty_batch(g, oracle_lib):
    import torch

    code, _, _ = code_pair(g, oracle_lib, 128)
    p = g.Params.make(M=16, S=10)
    r = g.decode_symbols(code, p, torch.zeros((0, 32), dtype=torch.complex64, device="cuda"), stats=True)
    torch.cuda.synchronize()
    assert r["cw"].shape == (0, 4) and r["hard_frames"] == 0


def test_nonfinite_frames(g, oracle_lib):
    N, M = 128, 16
    code, H, info = code_pair(g, oracle_lib, N)
    d = wl.qam_frames(33, 0, 40, N, info, M, 8.0)
    s = d["symbols"].copy()
    s[3, 4] = np.complex64(complex(np.nan, 1.0))
    s[17, 31] = np.complex64(complex(-np.inf, 0.0))
    want = oracle_lib.decode_qam(H, s, M, 10, 1 << 20, threads=THREADS)
    got = gpu_decode(g, code, s, M, 10, 1 << 20)
    assert_same(got, want)
    assert got["abandon"][3] == 2 and got["abandon"][17] == 2


def test_statistics_are_consistent(g, oracle_lib):
    N, M, S = 128, 16, 10
    code, H, info = code_pair(g, oracle_lib, N)
    d = wl.qam_frames(34, 0, 400, N, info, M, 6.0)
    got = gpu_decode(g, code, d["symbols"], M, S, 1 << 20, stats=True)
    useful = int(got["queries"].sum())
    assert got["evaluated_checks"] >= useful
    assert 0 < got["hard_frames"] <= 400


# ---------------------------------------------------------------------------
# bit-level GRAND-AB (the N=32 BPSK workload: 10,000 frames at 4 dB)
# ---------------------------------------------------------------------------

def test_grand_ab_full_workload(g, oracle_lib):
    import torch

    N = 32
    code, H, info = code_pair(g, oracle_lib, N)
    d = wl.bpsk_frames(1, 0, 10000, N, info, 4.0)
    want = oracle_lib.decode_ab(H, d["symbols"], 3, 5489, threads=THREADS)
    p = g.Params.make(order=g.ORDER_HAMMING, M=2, max_weight=3, query_cap=5489)
    r = g.decode_symbols(code, p, to_dev(d["symbols"]))
    torch.cuda.synchronize()
    got = {"cw": u32(r["cw"]), "queries": u32(r["queries"]).astype(np.int64), "abandon": r["abandon"].cpu().numpy()}
    assert_same(got, want, "GRAND-AB")
    # the two-call path (hard word from grand_demod) agrees
    dm = g.demod(to_dev(d["symbols"]), 2, N)
    r2 = g.decode_batch(code, p, dm["y"], nmask=dm["nmask"])
    torch.cuda.synchronize()
    assert torch.equal(r2["cw"], r["cw"]) and torch.equal(r2["queries"], r["queries"])


@pytest.mark.parametrize("N,w,cap", [(64, 4, 10 ** 6), (128, 2, 3000), (256, 3, 20000)])
def test_grand_ab_other_sizes(g, oracle_lib, N, w, cap):
    import torch

    code, H, info = code_pair(g, oracle_lib, N)
    d = wl.bpsk_frames(2, N, 200, N, info, 5.0)
    want = oracle_lib.decode_ab(H, d["symbols"], w, cap, threads=THREADS)
    p = g.Params.make(order=g.ORDER_HAMMING, M=2, max_weight=w, query_cap=cap)
    r = g.decode_symbols(code, p, to_dev(d["symbols"]))
    torch.cuda.synchronize()
    got = {"cw": u32(r["cw"]), "queries": u32(r["queries"]).astype(np.int64), "abandon": r["abandon"].cpu().numpy()}
    assert_same(got, want, f"AB N={N}")


@pytest.mark.parametrize("N,K,w,cap,snr", [
    (32, 16, 3, 1000, 3.0),      # cap inside the weight-3 class
    (32, 16, 2, 529, 3.0),       # weights <= 2 only, the whole space
    (32, 16, 1, 20, 6.0),        # cap inside the weight-1 class
    (32, 8, 3, 5489, 2.0),       # 24 parity bits (the 32-plane compare)
    (32, 12, 3, 5489, 1.0),      # 20 parity bits, low SNR: many weight-3 hits and abandons
    (64, 32, 3, 10 ** 6, 4.0),   # two 32-position groups, 32 parity bits
    (64, 48, 3, 45000, 5.0),     # two groups, 16 parity bits
])
def test_grand_ab_split_kernel(g, oracle_lib, N, K, w, cap, snr):
    """The pair x single split of the bit-level search (N <= 64, N - K <= 32,
    weights <= 3) against the oracle's sequential walk, including caps that
    cut a weight class and codes with few and many parity bits."""
    import torch

    code, H, info = code_pair(g, oracle_lib, N, K)
    d = wl.bpsk_frames(9, N * 100 + K, 3000, N, info, snr)
    want = oracle_lib.decode_ab(H, d["symbols"], w, cap, threads=THREADS)
    p = g.Params.make(order=g.ORDER_HAMMING, M=2, max_weight=w, query_cap=cap)
    r = g.decode_symbols(code, p, to_dev(d["symbols"]))
    torch.cuda.synchronize()
    got = {"cw": u32(r["cw"]), "queries": u32(r["queries"]).astype(np.int64), "abandon": r["abandon"].cpu().numpy()}
    assert_same(got, want, f"AB split N={N} K={K} w={w} cap={cap}")


# ---------------------------------------------------------------------------
# uneven batch
# ---------------------------------------------------------------------------

def test_mixed_batch_parity(g, oracle_lib):
    import torch

    Ns = (32, 64, 128, 256)
    codes = [code_pair(g, oracle_lib, n)[0] for n in Ns]
    info = {n: code_pair(g, oracle_lib, n)[2] for n in Ns}
    mx = wl.mixed_frames(40, 0, 600, info, ebn0_range=(8.0, 14.0), n_choices=Ns)
    code_idx = np.searchsorted(np.array(Ns), mx["N"])
    desc = g.frame_desc(code_idx, mx["M"], mx["sym_offset"], mx["cw_offset"])
    p = g.Params.make(M=0, S=8, query_cap=1 << 16)
    r = g.decode_mixed(codes, p, to_dev(desc.view(np.uint8)), to_dev(mx["symbols"]), mx["n_cw_words"])
    torch.cuda.synchronize()
    cw, q, ab = u32(r["cw"]), u32(r["queries"]).astype(np.int64), r["abandon"].cpu().numpy()
    for n in Ns:
        for M in wl.QAM_ORDERS:
            idx = np.nonzero((mx["N"] == n) & (mx["M"] == M))[0]
            if idx.size == 0:
                continue
            L = wl.symbols_per_frame(n, M)
            sym = np.stack([mx["symbols"][mx["sym_offset"][f]:mx["sym_offset"][f] + L] for f in idx])
            want = oracle_lib.decode_qam(code_pair(g, oracle_lib, n)[1], sym, M, 8, 1 << 16, threads=THREADS)
            got = {"cw": np.stack([cw[mx["cw_offset"][f]:mx["cw_offset"][f] + n // 32] for f in idx]),
                   "queries": q[idx], "abandon": ab[idx]}
            assert_same(got, want, f"mixed N={n} M={M}")


@pytest.mark.parametrize("membership", [0, 3])
def test_mixed_batch_s12(g, oracle_lib, membership):
    """S = 12 over an uneven batch: frames of every S' from 3 to 12 go through
    the warp search (or the hash join with 6-rank sides) in one launch."""
    import torch

    Ns = (32, 64, 128, 256)
    codes = [code_pair(g, oracle_lib, n)[0] for n in Ns]
    info = {n: code_pair(g, oracle_lib, n)[2] for n in Ns}
    mx = wl.mixed_frames(42, membership, 400, info, ebn0_range=(9.0, 14.0), n_choices=Ns)
    code_idx = np.searchsorted(np.array(Ns), mx["N"])
    desc = g.frame_desc(code_idx, mx["M"], mx["sym_offset"], mx["cw_offset"])
    p = g.Params.make(M=0, S=12, query_cap=1 << 18, membership=membership)
    r = g.decode_mixed(codes, p, to_dev(desc.view(np.uint8)), to_dev(mx["symbols"]), mx["n_cw_words"])
    torch.cuda.synchronize()
    cw, q, ab = u32(r["cw"]), u32(r["queries"]).astype(np.int64), r["abandon"].cpu().numpy()
    for n in Ns:
        for M in wl.QAM_ORDERS:
            idx = np.nonzero((mx["N"] == n) & (mx["M"] == M))[0][:12]
            if idx.size == 0:
                continue
            L = wl.symbols_per_frame(n, M)
            sym = np.stack([mx["symbols"][mx["sym_offset"][f]:mx["sym_offset"][f] + L] for f in idx])
            want = oracle_lib.decode_qam(code_pair(g, oracle_lib, n)[1], sym, M, 12, 1 << 18, threads=THREADS)
            got = {"cw": np.stack([cw[mx["cw_offset"][f]:mx["cw_offset"][f] + n // 32] for f in idx]),
                   "queries": q[idx], "abandon": ab[idx]}
            assert_same(got, want, f"mixed S=12 N={n} M={M}")


def test_mixed_rejects_bad_descriptors(g, oracle_lib):
    import torch

    code = code_pair(g, oracle_lib, 128)[0]
    sym = torch.zeros(64, dtype=torch.complex64, device="cuda")
    desc = g.frame_desc([0, 1, 0, 0], [16, 16, 8, 16], [0, 0, 0, 40], [0, 4, 8, 12])
    p = g.Params.make(M=0, S=8, query_cap=100)
    r = g.decode_mixed([code], p, to_dev(desc.view(np.uint8)), sym, 16)
    torch.cuda.synchronize()
    ab = r["abandon"].cpu().tolist()
    assert ab[1:] == [3, 3, 3] and ab[0] in (0, 1)


@pytest.mark.parametrize("N,M,S", [(128, 16, 10), (512, 64, 8), (1024, 256, 12)])
def test_general_H_path_matches_polar_path(g, oracle_lib, N, M, S):
    """The same code given by a parity-check matrix that is not in polar form
    (row 0 replaced by row 0 xor row 1: same null space) takes the general
    column path; its decisions must equal those of the polar-form matrix."""
    import torch

    code, H, info = code_pair(g, oracle_lib, N)
    Hp, _ = g.polar_H(N, N // 2)
    Hg = Hp.copy()
    Hg[0] ^= Hg[1]
    code_g = g.Code(Hg, N, N // 2)
    d = wl.qam_frames(41, N + M, 300, N, info, M, 10.0 if M < 256 else 16.0)
    cap = 1 << 16
    a = gpu_decode(g, code, d["symbols"], M, S, cap)
    b = gpu_decode(g, code_g, d["symbols"], M, S, cap)
    assert_same(b, a, "general vs polar H")
    Hd = H.copy()
    Hd[0] ^= Hd[1]
    want = oracle_lib.decode_qam(Hd, d["symbols"][:60], M, S, cap, threads=THREADS)
    assert_same({k: v[:60] for k, v in b.items()}, want, "general H vs oracle")
    code_g.close()
