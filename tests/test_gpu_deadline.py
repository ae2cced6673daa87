"""The watchdog: grand_params.deadline_ns and grand_stream_status.

A frame that a search warp fetches after the call's budget ran out is not
searched: abandon 5, cw = the hard word, queries = the valid TEPs already tested
without a hit (the preparation's: every TEP with at most two altered symbols;
none for the per-TEP and bit-level kernels). Every other frame must equal the
oracle, and the code's status word must report the cut exactly once."""
from __future__ import annotations

import numpy as np
import pytest

import workloads as wl

pytestmark = pytest.mark.gpu

N, K, M = 128, 64, 16


@pytest.fixture(scope="module")
def g():
    import torch

    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2405_01808_gb300 as grand

    grand.build()
    return grand


def prep_tested(oracle_lib, sym, M, N, S, w0=2):
    """Valid TEPs with at most w0 altered symbols among the S' least reliable:
    e_0 + ... + e_w0 of the alternative counts (Cor. III.1's count by weight)."""
    dm = oracle_lib.demod(sym, M, N)
    out = np.zeros(sym.shape[0], np.int64)
    for f in range(sym.shape[0]):
        sel = oracle_lib.select(dm["key"][f], S)
        k = np.array([bin(int(v) & 7).count("1") for v in dm["nmask"][f][sel]], np.int64)
        e = np.zeros(w0 + 1, np.int64)
        e[0] = 1
        for kv in k:  # multiply the generating polynomial by (1 + k x)
            e[1:] = e[1:] + kv * e[:-1]
        out[f] = e.sum()
    return out, dm["y"]


def check_cut_or_oracle(oracle_lib, H, sym, cw, q, ab, M, S, cap, order=1, tested=None, y=None):
    cut = ab == 5
    keep = ~cut
    if keep.any():
        want = oracle_lib.decode_qam(H, sym[keep], M, S, cap, order=order, threads=8)
        assert np.array_equal(cw[keep], want["cw"])
        assert np.array_equal(q[keep], want["queries"])
        assert np.array_equal(ab[keep], want["abandon"])
    if cut.any():
        if y is None:
            y = oracle_lib.demod(sym[cut], M, N)["y"]
        else:
            y = y[cut]
        assert np.array_equal(cw[cut], y)
        if tested is None:
            assert np.all(q[cut] == 0)
        else:
            assert np.array_equal(q[cut], tested[cut])
    return cut


@pytest.mark.parametrize("membership", [0, 3])
def test_expired_budget_cuts_every_searched_frame(g, oracle_lib, membership):
    """A 1 ns budget has run out before the search kernel starts: every frame
    the preparation hands on is cut, every frame it resolves is decoded."""
    import torch

    code = g.Code.polar(N, K)
    H = oracle_lib.parity_H(N, K)
    d = wl.qam_frames(2, 0, 3000, N, oracle_lib.info_set(N, K), M, 6.0)
    sym = d["symbols"]
    S, cap = 10, 1 << 20
    p = g.Params.make(M=M, S=S, query_cap=cap, membership=membership, deadline_ns=1)
    r = g.decode_symbols(code, p, torch.from_numpy(sym).cuda(), stats=True)
    assert g.stream_status(code) == g.E_TIMEOUT
    assert g.stream_status(code) == 0  # taken and cleared
    cw = r["cw"].cpu().numpy().view(np.uint32)
    q = r["queries"].cpu().numpy().astype(np.int64)
    ab = r["abandon"].cpu().numpy()
    tested, y = prep_tested(oracle_lib, sym, M, N, S)
    cut = check_cut_or_oracle(oracle_lib, H, sym, cw, q, ab, M, S, cap, tested=tested, y=y)
    assert int(cut.sum()) == int(r["hard_frames"]) > 100
    # the same batch without a budget: identical outside the cut frames, and
    # the cut frames needed more queries than the preparation's
    r0 = g.decode_symbols(code, g.Params.make(M=M, S=S, query_cap=cap, membership=membership),
                          torch.from_numpy(sym).cuda())
    assert g.stream_status(code) == 0
    q0 = r0["queries"].cpu().numpy().astype(np.int64)
    assert np.all(q0[cut] > tested[cut])
    if membership == 0:
        # the fixed-scratch entry and a captured plan (the clock restarts at
        # every replay) cut the same frames
        x = torch.from_numpy(sym).cuda()
        outs = [torch.empty_like(r["cw"]), torch.empty_like(r["queries"]), torch.empty_like(r["abandon"])]
        g.decode_symbols_noalloc(code, p, x, *outs)
        assert g.stream_status(code) == g.E_TIMEOUT
        for k, o in zip(("cw", "queries", "abandon"), outs):
            assert torch.equal(r[k], o), k
        outs = [torch.empty_like(r["cw"]), torch.empty_like(r["queries"]), torch.empty_like(r["abandon"])]
        plan = g.plan_symbols(code, p, x, *outs)
        assert g.stream_status(code) == g.E_TIMEOUT  # the eager run at creation
        for _ in range(2):
            for o in outs:
                o.zero_()
            plan.launch()
            assert g.stream_status(code) == g.E_TIMEOUT
            for k, o in zip(("cw", "queries", "abandon"), outs):
                assert torch.equal(r[k], o), k
        plan.close()
    code.close()


def test_generous_budget_changes_nothing(g, oracle_lib):
    import torch

    code = g.Code.polar(N, K)
    d = wl.qam_frames(2, 1, 4000, N, oracle_lib.info_set(N, K), M, 6.0)
    x = torch.from_numpy(d["symbols"]).cuda()
    base = g.decode_symbols(code, g.Params.make(M=M, S=10, query_cap=1 << 20), x)
    for order, membership in ((1, 0), (1, 3), (2, 0), (3, 0), (1, 1)):
        a = g.decode_symbols(code, g.Params.make(order=order, M=M, S=10, query_cap=1 << 20, membership=membership), x)
        b = g.decode_symbols(code, g.Params.make(order=order, M=M, S=10, query_cap=1 << 20, membership=membership,
                                                 deadline_ns=10 ** 10), x)
        for k in ("cw", "queries", "abandon"):
            assert torch.equal(a[k], b[k]), (order, membership, k)
        assert int((b["abandon"] == 5).sum()) == 0
        assert g.stream_status(code) == 0
    del base
    code.close()


@pytest.mark.parametrize("order,membership", [(3, 0), (1, 2)])
def test_per_tep_kernel_cuts_late_frames(g, oracle_lib, order, membership):
    """The per-TEP kernel has no preparation stage: a frame fetched after the
    budget is the hard word with queries 0; the rest equal the oracle."""
    import torch

    code = g.Code.polar(N, K)
    H = oracle_lib.parity_H(N, K)
    d = wl.qam_frames(2, 2, 6000, N, oracle_lib.info_set(N, K), M, 6.0)
    sym = d["symbols"]
    S, cap = 8, 1 << 16
    p = g.Params.make(order=order, M=M, S=S, query_cap=cap, membership=membership, deadline_ns=1)
    r = g.decode_symbols(code, p, torch.from_numpy(sym).cuda())
    st = g.stream_status(code)
    ab = r["abandon"].cpu().numpy()
    assert st == (g.E_TIMEOUT if (ab == 5).any() else 0)
    oracle_order = 3 if order == 3 else 1
    cut = check_cut_or_oracle(oracle_lib, H, sym, r["cw"].cpu().numpy().view(np.uint32),
                              r["queries"].cpu().numpy().astype(np.int64), ab, M, S, cap, order=oracle_order)
    assert cut.sum() > 0  # 6000 frames outlast the first wave of warps
    code.close()


def test_bit_level_kernel_cuts_late_frames(g, oracle_lib):
    import torch

    Nb, Kb = 32, 16
    code = g.Code.polar(Nb, Kb)
    H = oracle_lib.parity_H(Nb, Kb)
    d = wl.bpsk_frames(1, 0, 20000, Nb, oracle_lib.info_set(Nb, Kb), 4.0)
    r_in = d["symbols"]
    p = g.Params.make(order=g.ORDER_HAMMING, M=2, S=0, max_weight=3, query_cap=5489, deadline_ns=1)
    r = g.decode_symbols(code, p, torch.from_numpy(r_in).cuda())
    ab = r["abandon"].cpu().numpy()
    assert g.stream_status(code) == (g.E_TIMEOUT if (ab == 5).any() else 0)
    assert (ab == 5).sum() > 0
    cw = r["cw"].cpu().numpy().view(np.uint32)
    q = r["queries"].cpu().numpy().astype(np.int64)
    keep = ab != 5
    want = oracle_lib.decode_ab(H, r_in[keep], 3, 5489, threads=8)
    assert np.array_equal(cw[keep], want["cw"]) and np.array_equal(q[keep], want["queries"])
    assert np.array_equal(ab[keep], want["abandon"])
    hard = wl.pack_bits((r_in[~keep] < 0).astype(np.uint8))
    assert np.array_equal(cw[~keep], hard) and np.all(q[~keep] == 0)
    code.close()


def test_mixed_batch_flags_the_codes_it_cut(g, oracle_lib):
    """An uneven batch over three codes: each code's status word reports
    whether one of its frames was cut."""
    import torch

    Ns = (32, 128, 512)
    codes = [g.Code.polar(n, n // 2) for n in Ns]
    parts, desc, sym_off, cw_off = [], [], 0, 0
    for i, n in enumerate(Ns):
        Mi = 4 if n == 32 else 16
        snr = 12.0 if n == 32 else 5.0  # the N=32 frames are all resolved by the preparation
        dd = wl.qam_frames(41, i, 400, n, oracle_lib.info_set(n, n // 2), Mi, snr)
        L = dd["symbols"].shape[1]
        for f in range(400):
            desc.append((i, Mi, sym_off + f * L, cw_off + f * (n // 32)))
        parts.append(dd["symbols"].reshape(-1))
        sym_off += 400 * L
        cw_off += 400 * (n // 32)
    desc_np = g.frame_desc(*map(np.array, zip(*desc)))
    sym = np.concatenate(parts).astype(np.complex64)
    p = g.Params.make(M=16, S=10, query_cap=1 << 20, deadline_ns=1)
    r = g.decode_mixed(codes, p, torch.from_numpy(desc_np.view(np.uint8)).cuda(), torch.from_numpy(sym).cuda(), cw_off)
    torch.cuda.synchronize()
    ab = r["abandon"].cpu().numpy()
    for i in range(3):
        any_cut = bool((ab[400 * i:400 * (i + 1)] == 5).any())
        assert g.stream_status(codes[i]) == (g.E_TIMEOUT if any_cut else 0), i
    assert not (ab[:400] == 5).any() and (ab[400:] == 5).any()
    for c in codes:
        c.close()


def test_negative_budget_is_invalid(g):
    import torch

    code = g.Code.polar(N, K)
    x = torch.zeros(4, 32, dtype=torch.complex64, device="cuda")
    with pytest.raises(g.GrandError) as e:
        g.decode_symbols(code, g.Params.make(M=M, S=10, deadline_ns=-1), x)
    assert e.value.status == -1
    code.close()
