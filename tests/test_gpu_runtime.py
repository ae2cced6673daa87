"""GPU tests of the runtime around the kernels: CUDA-graph plans and the
launch-shape autotuner. Results must be bit-identical to the direct calls."""
from __future__ import annotations

import os

import numpy as np
import pytest

import workloads as wl

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def g():
    import torch

    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2405_01808_gb300 as grand

    grand.build()
    return grand


def info_of(g, N):
    _, frozen = g.polar_H(N, N // 2)
    return np.setdiff1d(np.arange(N), frozen)


def test_plan_symbols_replays_on_new_inputs(g):
    import torch

    N, M = 128, 16
    code = g.Code.polar(N, N // 2)
    p = g.Params.make(M=M, S=10, query_cap=1 << 20)
    batches = [wl.qam_frames(50, k, 3000, N, info_of(g, N), M, 6.0 + 2 * k)["symbols"] for k in range(3)]
    sym = torch.from_numpy(batches[0]).cuda()
    cw = torch.empty((3000, N // 32), dtype=torch.int32, device="cuda")
    q = torch.empty(3000, dtype=torch.int32, device="cuda")
    ab = torch.empty(3000, dtype=torch.uint8, device="cuda")
    plan = g.plan_symbols(code, p, sym, cw, q, ab)
    for b in batches:
        sym.copy_(torch.from_numpy(b))
        plan.launch()
        ref = g.decode_symbols(code, p, torch.from_numpy(b).cuda())
        torch.cuda.synchronize()
        assert torch.equal(cw, ref["cw"]) and torch.equal(q, ref["queries"]) and torch.equal(ab, ref["abandon"])
    plan.close()


def test_plan_mixed_matches_direct(g):
    import torch

    Ns = (32, 64, 128, 256, 512, 1024)
    codes = [g.Code.polar(n, n // 2) for n in Ns]
    mx = wl.mixed_frames(51, 0, 4000, {n: info_of(g, n) for n in Ns})
    desc = torch.from_numpy(g.frame_desc(np.searchsorted(np.array(Ns), mx["N"]), mx["M"], mx["sym_offset"],
                                         mx["cw_offset"]).view(np.uint8)).cuda()
    sym = torch.from_numpy(mx["symbols"]).cuda()
    p = g.Params.make(M=0, S=10, query_cap=1 << 20)
    cw = torch.empty(mx["n_cw_words"], dtype=torch.int32, device="cuda")
    q = torch.empty(4000, dtype=torch.int32, device="cuda")
    ab = torch.empty(4000, dtype=torch.uint8, device="cuda")
    plan = g.plan_mixed(codes, p, desc, sym, cw, q, ab)
    plan.launch()
    plan.launch()  # replay on the same inputs: same outputs
    ref = g.decode_mixed(codes, p, desc, sym, mx["n_cw_words"])
    torch.cuda.synchronize()
    assert torch.equal(cw, ref["cw"]) and torch.equal(q, ref["queries"]) and torch.equal(ab, ref["abandon"])
    plan.close()


def test_autotune_keeps_results_and_caches(g, tmp_path):
    import torch

    N, M = 128, 16
    code = g.Code.polar(N, N // 2)
    d = wl.qam_frames(52, 0, 4000, N, info_of(g, N), M, 7.0)
    sym = torch.from_numpy(d["symbols"]).cuda()
    p = g.Params.make(M=M, S=10, query_cap=1 << 20)
    cache = str(tmp_path / "tiles.txt")
    r1 = g.autotune(code, p, sym, cache_path=cache)
    assert not r1["from_cache"] and r1["candidates"] >= 2 and r1["best_ms"] > 0
    tuned = tuple(p.tiles)
    assert os.path.exists(cache)
    p2 = g.Params.make(M=M, S=10, query_cap=1 << 20)
    r2 = g.autotune(code, p2, sym, cache_path=cache)
    assert r2["from_cache"] and tuple(p2.tiles) == tuned
    a = g.decode_symbols(code, p, sym)
    b = g.decode_symbols(code, g.Params.make(M=M, S=10, query_cap=1 << 20), sym)
    torch.cuda.synchronize()
    assert torch.equal(a["cw"], b["cw"]) and torch.equal(a["queries"], b["queries"])


def test_autotune_mixed(g):
    import torch

    Ns = (64, 256)
    codes = [g.Code.polar(n, n // 2) for n in Ns]
    mx = wl.mixed_frames(53, 0, 2000, {n: info_of(g, n) for n in Ns}, n_choices=Ns)
    desc = torch.from_numpy(g.frame_desc(np.searchsorted(np.array(Ns), mx["N"]), mx["M"], mx["sym_offset"],
                                         mx["cw_offset"]).view(np.uint8)).cuda()
    sym = torch.from_numpy(mx["symbols"]).cuda()
    p = g.Params.make(M=0, S=10, query_cap=1 << 20)
    r = g.autotune_mixed(codes, p, desc, sym, mx["n_cw_words"])
    assert r["candidates"] >= 2
    a = g.decode_mixed(codes, p, desc, sym, mx["n_cw_words"])
    b = g.decode_mixed(codes, g.Params.make(M=0, S=10, query_cap=1 << 20), desc, sym, mx["n_cw_words"])
    torch.cuda.synchronize()
    assert torch.equal(a["cw"], b["cw"]) and torch.equal(a["queries"], b["queries"])


@pytest.mark.parametrize("S,N,M,snr", [(10, 128, 16, 7.0), (12, 512, 64, 14.0)])
def test_autotune_chooses_membership(g, tmp_path, S, N, M, snr):
    """GRAND_MEMBERSHIP_FASTEST: the tuner times both exact membership tests
    with their launch shapes, writes the faster into params.membership, records
    it in the cache, and the tuned decode equals the TEP-by-TEP one."""
    import torch

    code = g.Code.polar(N, N // 2)
    d = wl.qam_frames(54, S, 3000, N, info_of(g, N), M, snr)
    sym = torch.from_numpy(d["symbols"]).cuda()
    p = g.Params.make(M=M, S=S, query_cap=1 << 20, membership=g.MEMBERSHIP_FASTEST)
    cache = str(tmp_path / "tiles.txt")
    r = g.autotune(code, p, sym, cache_path=cache)
    assert p.membership in (g.MEMBERSHIP_AUTO, g.MEMBERSHIP_HASH) and r["membership"] == p.membership
    assert r["candidates"] > len({0, 3})  # shapes of both tests
    with open(cache) as fh:
        fields = fh.read().split()
    assert int(fields[-1]) == p.membership
    p2 = g.Params.make(M=M, S=S, query_cap=1 << 20, membership=g.MEMBERSHIP_FASTEST)
    r2 = g.autotune(code, p2, sym, cache_path=cache)
    assert r2["from_cache"] and p2.membership == p.membership and tuple(p2.tiles) == tuple(p.tiles)
    a = g.decode_symbols(code, p, sym)
    b = g.decode_symbols(code, g.Params.make(M=M, S=S, query_cap=1 << 20), sym)
    torch.cuda.synchronize()
    assert torch.equal(a["cw"], b["cw"]) and torch.equal(a["queries"], b["queries"])
    assert torch.equal(a["abandon"], b["abandon"])
    code.close()


@pytest.mark.parametrize("S,N,M,snr,warps", [(10, 128, 16, 7.0, (2, 4)), (12, 512, 64, 14.0, (1, 2))])
def test_autotune_hash_join_alone(g, S, N, M, snr, warps):
    """With membership HASH the tuner times the hash join's own launch shapes
    (warps per CTA x preparation weights, 6 candidates) and every candidate
    is a valid shape; the tuned decode equals the TEP-by-TEP one."""
    import torch

    code = g.Code.polar(N, N // 2)
    d = wl.qam_frames(55, S, 2000, N, info_of(g, N), M, snr)
    sym = torch.from_numpy(d["symbols"]).cuda()
    p = g.Params.make(M=M, S=S, query_cap=1 << 20, membership=g.MEMBERSHIP_HASH)
    r = g.autotune(code, p, sym)
    assert r["membership"] == g.MEMBERSHIP_HASH and r["candidates"] == 6 and not r["from_cache"]
    assert p.tiles[0] in warps and p.tiles[1] == 0 and p.tiles[2] in (1, 2, 3)
    a = g.decode_symbols(code, p, sym)
    b = g.decode_symbols(code, g.Params.make(M=M, S=S, query_cap=1 << 20), sym)
    torch.cuda.synchronize()
    assert torch.equal(a["cw"], b["cw"]) and torch.equal(a["queries"], b["queries"])
    assert torch.equal(a["abandon"], b["abandon"])
    code.close()
