"""Resumable decoding: a frame's TEP search run in windows of TEP weights with
its state (a cursor) kept in device memory between calls gives exactly the
outputs of the uninterrupted search (Alg. 2 Step 5: the TEPs come by weight in
the canonical order, so after every TEP of weight <= w is tested without a hit
the first hit of the rest is the first hit overall). Checked bit-exactly for
both membership tests (the TEP-by-TEP split search and the hash join), for
several window sizes, against grand_decode_symbols."""
from __future__ import annotations

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


CASES = [
    # N, M, S, cap, frames, Eb/N0, weight step
    (128, 16, 10, 1 << 20, 3000, 6.5, 1),
    (128, 16, 10, 1 << 20, 3000, 6.5, 3),
    (128, 16, 10, 5000, 3000, 6.5, 1),      # the cap falls inside weight class 4
    (512, 64, 12, 1 << 24, 1200, 13.0, 2),  # 5 + 7 ranks
    (1024, 256, 12, 1 << 20, 600, 16.0, 4),
]


@pytest.mark.parametrize("membership", [0, 3])
@pytest.mark.parametrize("N,M,S,cap,F,snr,step", CASES)
def test_split_and_resume_equals_uninterrupted(g, membership, N, M, S, cap, F, snr, step):
    import torch

    code = g.Code.polar(N, N // 2)
    try:
        _, frozen = g.polar_H(N, N // 2)
        info = np.setdiff1d(np.arange(N), frozen)
        d = wl.qam_frames(90, N + step, F, N, info, M, snr)
        sym = torch.from_numpy(d["symbols"]).cuda()
        p = g.Params.make(M=M, S=S, query_cap=cap, membership=membership)
        ref = g.decode_symbols(code, p, sym)
        r = g.decode_symbols_resumable(code, p, sym, step)
        torch.cuda.synchronize()
        sus = r["abandon"] == g.ABANDON_SUSPENDED
        assert int(sus.sum()) > 0, "the first window suspends some frames"
        # frames finished in the first window already equal the uninterrupted outputs
        fin = ~sus
        assert torch.equal(r["queries"][fin], ref["queries"][fin]) and torch.equal(r["abandon"][fin], ref["abandon"][fin])
        # a suspended frame reports the TEPs tested so far, never more than its final count
        assert bool((r["queries"][sus].to(torch.int64) <= ref["queries"][sus].to(torch.int64)).all())
        assert bool((r["queries"][sus].to(torch.int64) < ref["queries"][sus].to(torch.int64) + 1).all())
        rounds = 0
        prev = r["queries"].clone()
        while bool((r["abandon"] == g.ABANDON_SUSPENDED).any()):
            rounds += 1
            assert rounds <= S, "every window advances the tested weight"
            g.decode_resume(code, p, r["cursors"], r["cw"], r["queries"], r["abandon"], weight_step=step)
            torch.cuda.synchronize()
            # the tested count only grows
            assert bool((r["queries"].to(torch.int64) >= prev.to(torch.int64)).all())
            prev = r["queries"].clone()
        assert rounds >= 1
        assert torch.equal(r["cw"], ref["cw"])
        assert torch.equal(r["queries"], ref["queries"])
        assert torch.equal(r["abandon"], ref["abandon"])
    finally:
        torch.cuda.synchronize()
        code.close()


def test_resume_rest_in_one_call(g):
    """A first window of one weight, then every remaining weight at once
    (weight_step 0): the same outputs."""
    import torch

    N, M = 128, 16
    code = g.Code.polar(N, N // 2)
    try:
        _, frozen = g.polar_H(N, N // 2)
        info = np.setdiff1d(np.arange(N), frozen)
        d = wl.qam_frames(91, 0, 2000, N, info, M, 7.0)
        sym = torch.from_numpy(d["symbols"]).cuda()
        p = g.Params.make(M=M, S=10, query_cap=1 << 20)
        ref = g.decode_symbols(code, p, sym)
        r = g.decode_symbols_resumable(code, p, sym, 1)
        g.decode_resume(code, p, r["cursors"], r["cw"], r["queries"], r["abandon"], weight_step=0)
        torch.cuda.synchronize()
        assert not bool((r["abandon"] == g.ABANDON_SUSPENDED).any())
        assert torch.equal(r["cw"], ref["cw"]) and torch.equal(r["queries"], ref["queries"])
        assert torch.equal(r["abandon"], ref["abandon"])
    finally:
        torch.cuda.synchronize()
        code.close()


def test_resumable_argument_checks(g):
    import torch

    code = g.Code.polar(128, 64)
    try:
        sym = torch.zeros((4, 32), dtype=torch.complex64, device="cuda")
        p = g.Params.make(M=16, S=10, query_cap=1 << 20)
        with pytest.raises(g.GrandError) as e:
            g.decode_symbols_resumable(code, p, sym, 0)  # the first call needs a window
        assert e.value.status == -1
        ps = g.Params.make(M=16, S=10, query_cap=1 << 20, tiles=(0, 5, 0, 0))  # explicit split
        with pytest.raises(g.GrandError) as e:
            g.decode_symbols_resumable(code, ps, sym, 1)
        assert e.value.status == -7
        pn = g.Params.make(order=g.ORDER_QAM_NNE5, M=16, S=8, query_cap=1 << 20)
        with pytest.raises(g.GrandError) as e:
            g.decode_symbols_resumable(code, pn, sym, 1)
        assert e.value.status == -7
    finally:
        code.close()
