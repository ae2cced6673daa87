"""GRAND_MEMBERSHIP_SOLVE on the GPU: the first hit of Alg. 2 Step 5 found by
Gaussian elimination over the frame's TEP coordinates (the reading pinned in
test_solve_reading.py) instead of a test per TEP. Decoded words, query
counts and abandon flags must equal the oracle's canonical walk: on the
parity cases of the split search, with the nearer-axis order and the literal
likelihood, on uneven batches, through the serving loop, and on every stored
frame of the full-size workloads."""
from __future__ import annotations

import numpy as np
import pytest

import workloads as wl
from test_gpu_fullsize import UNIFORM, check_properties, compare_stratum, load_golden
from test_gpu_parity import CASES, THREADS, assert_same, code_pair, to_dev, u32

pytestmark = pytest.mark.gpu

SOLVE = 5
NNE, NEARER, NNE5 = 1, 2, 3


@pytest.fixture(scope="module")
def g():
    import torch

    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2405_01808_gb300 as grand

    grand.build()
    assert grand.MEMBERSHIP_SOLVE == SOLVE
    return grand


def unpack(r):
    import torch

    torch.cuda.synchronize()
    return {"cw": u32(r["cw"]), "queries": u32(r["queries"]).astype(np.int64), "abandon": r["abandon"].cpu().numpy()}


@pytest.mark.parametrize("N,M,S,snr,cap,F,lik", CASES)
def test_solve_parity(g, oracle_lib, N, M, S, snr, cap, F, lik):
    code, H, info = code_pair(g, oracle_lib, N)
    d = wl.qam_frames(20 + N, int(snr * 10) + S, F, N, info, M, snr)
    want = oracle_lib.decode_qam(H, d["symbols"], M, S, cap, literal=bool(lik), threads=THREADS)
    p = g.Params.make(M=M, S=S, query_cap=cap, lik_variant=lik, membership=SOLVE)
    got = unpack(g.decode_symbols(code, p, to_dev(d["symbols"])))
    assert_same(got, want, f"solve N={N} M={M} S={S}")


@pytest.mark.parametrize("N,M,S,snr,cap,F,lik", [
    (128, 16, 10, 7.0, 1 << 20, 300, 0),
    (256, 64, 9, 10.0, 4 ** 9, 200, 0),
    (32, 4, 8, 3.0, 1 << 16, 300, 0),
    (128, 16, 10, 7.0, 1 << 20, 200, 1),
    (1024, 256, 12, 15.0, 1 << 24, 60, 0),
])
def test_solve_nearer_order(g, oracle_lib, N, M, S, snr, cap, F, lik):
    code, H, info = code_pair(g, oracle_lib, N)
    d = wl.qam_frames(70, N + M + S, F, N, info, M, snr)
    want = oracle_lib.decode_qam(H, d["symbols"], M, S, cap, literal=bool(lik), threads=THREADS, order=NEARER)
    p = g.Params.make(order=NEARER, M=M, S=S, query_cap=cap, lik_variant=lik, membership=SOLVE)
    got = unpack(g.decode_symbols(code, p, to_dev(d["symbols"])))
    assert_same(got, want, f"solve nearer N={N} M={M} S={S}")


def test_solve_two_call_path_and_stats(g, oracle_lib):
    """grand_decode_batch on grand_demod's arrays equals the fused call; the
    statistics count the ranked solutions and hand no frame of this batch
    to the TEP search (kernel dimensions stay small)."""
    import torch

    N, M, S = 128, 16, 10
    code, H, info = code_pair(g, oracle_lib, N)
    d = wl.qam_frames(71, 3, 4000, N, info, M, 7.0)
    sym = to_dev(d["symbols"])
    p = g.Params.make(M=M, S=S, query_cap=1 << 20, membership=SOLVE)
    fused = g.decode_symbols(code, p, sym, stats=True)
    a = unpack(fused)
    dm = g.demod(sym, M, N)
    b = unpack(g.decode_batch(code, p, dm["y"], dm["hard_idx"], dm["key"], dm["nmask"]))
    assert_same(b, a, "two-call solve")
    want = oracle_lib.decode_qam(H, d["symbols"][:800], M, S, 1 << 20, threads=THREADS)
    assert_same({k: v[:800] for k, v in a.items()}, want, "solve stats batch")
    assert fused["hard_frames"] == 0
    assert fused["evaluated_checks"] >= int((a["abandon"] == 0).sum())


def test_solve_plan_host_memory_and_deadline(g, oracle_lib):
    """SOLVE through a CUDA-graph plan, from host memory, and with a device-time
    budget: the outputs equal the direct call's (the preparation decides every
    frame, and frames the preparation decides are never cut)."""
    import torch

    N, M, S = 128, 16, 10
    code, H, info = code_pair(g, oracle_lib, N)
    d = wl.qam_frames(72, 5, 3000, N, info, M, 7.0)
    sym = to_dev(d["symbols"])
    p = g.Params.make(M=M, S=S, query_cap=1 << 20, membership=SOLVE)
    ref = unpack(g.decode_symbols(code, p, sym))
    cw = torch.empty((3000, N // 32), dtype=torch.int32, device="cuda")
    q = torch.empty(3000, dtype=torch.int32, device="cuda")
    ab = torch.empty(3000, dtype=torch.uint8, device="cuda")
    plan = g.plan_symbols(code, p, sym, cw, q, ab)
    for _ in range(2):
        cw.zero_()
        q.zero_()
        ab.fill_(9)
        plan.launch()
        assert_same(unpack({"cw": cw, "queries": q, "abandon": ab}), ref, "solve plan")
    plan.close()
    h = g.decode_symbols_host(code, p, torch.from_numpy(d["symbols"]).pin_memory())
    assert_same({"cw": h["cw"].numpy().view(np.uint32), "queries": h["queries"].numpy().view(np.uint32).astype(np.int64),
                 "abandon": h["abandon"].numpy()}, ref, "solve host memory")
    pd = g.Params.make(M=M, S=S, query_cap=1 << 20, membership=SOLVE, deadline_ns=1)
    assert_same(unpack(g.decode_symbols(code, pd, sym)), ref, "solve with a deadline")


@pytest.mark.parametrize("S", [10, 12])
def test_solve_mixed_batch(g, oracle_lib, S):
    import torch

    Ns = (32, 64, 128, 256, 512)
    codes = [code_pair(g, oracle_lib, n)[0] for n in Ns]
    info = {n: code_pair(g, oracle_lib, n)[2] for n in Ns}
    mx = wl.mixed_frames(43, S, 600, info, ebn0_range=(6.0, 14.0), n_choices=Ns)
    code_idx = np.searchsorted(np.array(Ns), mx["N"])
    desc = g.frame_desc(code_idx, mx["M"], mx["sym_offset"], mx["cw_offset"])
    p = g.Params.make(M=0, S=S, query_cap=1 << 20, membership=SOLVE)
    r = g.decode_mixed(codes, p, to_dev(desc.view(np.uint8)), to_dev(mx["symbols"]), mx["n_cw_words"])
    torch.cuda.synchronize()
    cw, q, ab = u32(r["cw"]), u32(r["queries"]).astype(np.int64), r["abandon"].cpu().numpy()
    for n in Ns:
        for M in wl.QAM_ORDERS:
            idx = np.nonzero((mx["N"] == n) & (mx["M"] == M))[0][:16]
            if idx.size == 0:
                continue
            L = wl.symbols_per_frame(n, M)
            sym = np.stack([mx["symbols"][mx["sym_offset"][f]:mx["sym_offset"][f] + L] for f in idx])
            want = oracle_lib.decode_qam(code_pair(g, oracle_lib, n)[1], sym, M, S, 1 << 20, threads=THREADS)
            got = {"cw": np.stack([cw[mx["cw_offset"][f]:mx["cw_offset"][f] + n // 32] for f in idx]),
                   "queries": q[idx], "abandon": ab[idx]}
            assert_same(got, want, f"solve mixed S={S} N={n} M={M}")


def test_solve_refused_where_it_does_not_apply(g, oracle_lib):
    import torch

    N, M = 128, 16
    code, _, _ = code_pair(g, oracle_lib, N)
    sym = torch.zeros((4, 32), dtype=torch.complex64, device="cuda")
    with pytest.raises(g.GrandError) as e:  # five-point order: a fifth alternative per symbol
        g.decode_symbols(code, g.Params.make(order=NNE5, M=M, S=8, membership=SOLVE), sym)
    assert e.value.status == g.E_UNSUPPORTED
    r = torch.zeros((4, N), dtype=torch.float32, device="cuda")
    with pytest.raises(g.GrandError) as e:  # bit-level TEPs of bounded weight are not a coordinate space
        g.decode_symbols(code, g.Params.make(order=g.ORDER_HAMMING, M=2, S=0, max_weight=3, membership=SOLVE), r)
    assert e.value.status == g.E_UNSUPPORTED
    with pytest.raises(g.GrandError):  # the resumable search tests TEPs weight by weight
        g.decode_symbols_resumable(code, g.Params.make(M=M, S=8, membership=SOLVE), sym, weight_step=1)
    with pytest.raises(g.GrandError):  # the autotuner chooses among TEP-testing procedures
        g.autotune(code, g.Params.make(M=M, S=8, membership=SOLVE), sym)
    with pytest.raises(g.GrandError) as e:  # serving continuation resumes TEP searches
        g.Server([code], g.Params.make(M=0, S=8, membership=SOLVE), max_slots=16, max_device_bytes=1 << 20,
                 resume_weight_step=1)
    assert e.value.status == g.E_UNSUPPORTED


@pytest.mark.parametrize("config", ["c2", "c3a", "c3b"])
def test_solve_full_batch_equals_stored_outputs(g, oracle_lib, config):
    """The whole batch of each uniform workload through SOLVE; every stored
    frame equal to the oracle's (all 300,000 frames at N=128)."""
    import torch

    c = UNIFORM[config]
    z, meta = load_golden(config)
    N, K, M = c["N"], c["N"] // 2, c["M"]
    info = oracle_lib.info_set(N, K)
    parts = [wl.qam_frames(c["cid"], i, c["frames"], N, info, M, snr) for i, snr in enumerate(c["snrs"])]
    sym = np.concatenate([p["symbols"] for p in parts])
    code = g.Code.polar(N, K)
    try:
        p = g.Params.make(M=M, S=c["S"], query_cap=c["cap"], membership=SOLVE)
        r = g.decode_symbols(code, p, torch.from_numpy(sym).cuda())
        torch.cuda.synchronize()
        cw = r["cw"].cpu().numpy().view(np.uint32)
        q = r["queries"].cpu().numpy().view(np.uint32).astype(np.int64)
        ab = r["abandon"].cpu().numpy()
    finally:
        code.close()
    check_properties(oracle_lib.parity_H(N, K), cw, q, ab, oracle_lib.demod(sym, M, N)["y"], c["cap"])
    compared = 0
    for i in range(len(c["snrs"])):
        st = meta["strata"][f"s{i}"]
        lo = i * c["frames"]
        n, _ = compare_stratum(oracle_lib, z, f"s{i}", st, sym[lo:lo + c["frames"]], cw[lo:lo + c["frames"]],
                               q[lo:lo + c["frames"]], ab[lo:lo + c["frames"]])
        compared += n
    if config == "c2":
        assert compared == len(sym)


def test_solve_uneven_mix_equals_stored_outputs(g, oracle_lib):
    """The 1,000,000-frame uneven mix through SOLVE in one call; every stored
    frame of every (N, M) class equal to the oracle's."""
    import torch

    z, meta = load_golden("c4")
    Ns = wl.MIXED_N
    codes = [g.Code.polar(n, n // 2) for n in Ns]
    info = {n: oracle_lib.info_set(n, n // 2) for n in Ns}
    mx = wl.mixed_frames(5, 1000, 1000000, info)
    desc = torch.from_numpy(g.frame_desc(np.searchsorted(np.array(Ns), mx["N"]), mx["M"], mx["sym_offset"],
                                         mx["cw_offset"]).view(np.uint8)).cuda()
    p = g.Params.make(M=0, S=10, query_cap=1 << 20, membership=SOLVE)
    r = g.decode_mixed(codes, p, desc, torch.from_numpy(mx["symbols"]).cuda(), mx["n_cw_words"])
    torch.cuda.synchronize()
    cw = r["cw"].cpu().numpy().view(np.uint32)
    q = r["queries"].cpu().numpy().view(np.uint32).astype(np.int64)
    ab = r["abandon"].cpu().numpy()
    for c in codes:
        c.close()
    for n in Ns:
        for M in wl.QAM_ORDERS:
            f = np.nonzero((mx["N"] == n) & (mx["M"] == M))[0]
            L = wl.symbols_per_frame(n, M)
            symf = mx["symbols"][mx["sym_offset"][f][:, None] + np.arange(L)[None, :]]
            cwf = cw[mx["cw_offset"][f][:, None] + np.arange(n // 32)[None, :]]
            name = f"n{n}_m{M}"
            compare_stratum(oracle_lib, z, name, meta["strata"][name], symf, cwf, q[f], ab[f])
