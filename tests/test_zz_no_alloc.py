"""The allocation-free decode entry point (grand_decode_symbols_noalloc).

Some callers may not allocate device memory once they run (a receiver pipeline
that reserves everything at start-up, for instance). For them the library has
one extra call whose scratch is a fixed array inside the library instead of
stream-ordered allocations. These tests call it through the C ABI and require
results identical to grand_decode_symbols (integer outputs: bit-exact), on two
calls in a row with different batches, so that state left in the shared array
by the first call cannot leak into the second. The file is collected last."""
from __future__ import annotations

import ctypes

import numpy as np
import pytest

import workloads as wl

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    import torch

    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2405_01808_gb300 as g

    g.build()
    code = g.Code.polar(128, 64)
    _, frozen = g.polar_H(128, 64)
    info = np.setdiff1d(np.arange(128), frozen)
    yield g, code, info
    torch.cuda.synchronize()
    code.close()


def _call_noalloc(g, code, p, sym, F, words=4):
    """Call the entry point directly through ctypes (the C ABI)."""
    import torch

    cw = torch.full((F, words), -1, dtype=torch.int32, device="cuda")
    q = torch.full((F,), -1, dtype=torch.int32, device="cuda")
    ab = torch.full((F,), 255, dtype=torch.uint8, device="cuda")
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    rc = g.lib().grand_decode_symbols_noalloc(code.handle, ctypes.byref(p),
                                              ctypes.c_void_p(torch.view_as_real(sym).data_ptr()), F,
                                              ctypes.c_float(1.0), ctypes.c_void_p(cw.data_ptr()),
                                              ctypes.c_void_p(q.data_ptr()), ctypes.c_void_p(ab.data_ptr()), stream)
    assert rc == 0, g.lib().grand_status_string(rc)
    torch.cuda.synchronize()
    return cw, q, ab


def test_noalloc_matches_allocating_call_twice(env):
    import torch

    g, code, info = env
    p = g.Params.make(M=16, S=10, query_cap=1 << 20)
    # first call: a larger batch with many searched frames; second: a smaller
    # one, so stale records or counters from the first call would show
    batches = [wl.qam_frames(77, 0, 6000, 128, info, 16, 6.5), wl.qam_frames(77, 1, 2500, 128, info, 16, 9.0)]
    for d in batches:
        F = len(d["symbols"])
        sym = torch.from_numpy(d["symbols"]).cuda()
        ref = g.decode_symbols(code, p, sym)
        torch.cuda.synchronize()
        cw, q, ab = _call_noalloc(g, code, p, sym, F)
        assert torch.equal(cw, ref["cw"])
        assert torch.equal(q, ref["queries"])
        assert torch.equal(ab, ref["abandon"])
        assert int((ab == 1).sum()) > 0 and int((ab == 0).sum()) > 0


def test_noalloc_matches_allocating_call_s12(env):
    """S' = 12 (N=512, 64-QAM, cap 2^24): the search stage with a 7-rank B side,
    launched by the same helper as grand_decode_symbols; two calls in a row."""
    import torch

    g, _, _ = env
    N, K, M = 512, 256, 64
    code = g.Code.polar(N, K)
    try:
        _, frozen = g.polar_H(N, K)
        info = np.setdiff1d(np.arange(N), frozen)
        p = g.Params.make(M=M, S=12, query_cap=1 << 24)
        batches = [wl.qam_frames(78, 0, 1500, N, info, M, 14.0), wl.qam_frames(78, 1, 700, N, info, M, 15.0)]
        for d in batches:
            F = len(d["symbols"])
            sym = torch.from_numpy(d["symbols"]).cuda()
            ref = g.decode_symbols(code, p, sym)
            torch.cuda.synchronize()
            cw, q, ab = _call_noalloc(g, code, p, sym, F, N // 32)
            assert torch.equal(cw, ref["cw"])
            assert torch.equal(q, ref["queries"])
            assert torch.equal(ab, ref["abandon"])
            # frames decoded by the search stage (beyond the 631 TEPs of at most two
            # altered symbols that the preparation tests at S' = 12) are present
            assert int(((ab == 0) & (q.to(torch.int64) > 631)).sum()) > 0
    finally:
        torch.cuda.synchronize()
        code.close()


def test_noalloc_rejects_oversized_batch(env):
    import torch

    g, code, info = env
    p = g.Params.make(M=16, S=10, query_cap=1 << 20)
    F = g.NOALLOC_MAX_FRAMES + 1
    sym = torch.zeros((F, 32), dtype=torch.complex64, device="cuda")
    cw = torch.empty((F, 4), dtype=torch.int32, device="cuda")
    q = torch.empty(F, dtype=torch.int32, device="cuda")
    ab = torch.empty(F, dtype=torch.uint8, device="cuda")
    with pytest.raises(g.GrandError) as e:
        g.decode_symbols_noalloc(code, p, sym, cw, q, ab)
    assert e.value.status == -7  # GRAND_E_UNSUPPORTED
