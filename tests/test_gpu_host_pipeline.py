"""grand_decode_symbols_host: frames in host memory, chunks on two streams with
the copies overlapped. Its outputs must equal the device call's on the same
frames (which the parity tests pin to the oracle), for ragged chunkings,
pageable and page-locked buffers, both orders and both membership tests."""
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


def device_reference(g, code, p, sym):
    import torch

    r = g.decode_symbols(code, p, sym.cuda())
    torch.cuda.synchronize()
    return {k: r[k].cpu() for k in ("cw", "queries", "abandon")}


@pytest.mark.parametrize("chunk,pinned,membership", [(6000, True, 0), (7777, False, 0), (0, True, 3), (20000, True, 0)])
def test_equals_device_call(g, oracle_lib, chunk, pinned, membership):
    import torch

    N, K, M = 128, 64, 16
    code = g.Code.polar(N, K)
    d = wl.qam_frames(2, 5, 20000, N, oracle_lib.info_set(N, K), M, 7.0)
    sym = torch.from_numpy(d["symbols"])
    if pinned:
        sym = sym.pin_memory()
    p = g.Params.make(M=M, S=10, query_cap=1 << 20, membership=membership)
    want = device_reference(g, code, p, sym)
    got = g.decode_symbols_host(code, p, sym, chunk_frames=chunk)
    for k in ("cw", "queries", "abandon"):
        assert not got[k].is_cuda
        assert torch.equal(got[k], want[k]), k
    # a few frames against the oracle directly
    idx = np.arange(0, 20000, 997)
    o = oracle_lib.decode_qam(oracle_lib.parity_H(N, K), d["symbols"][idx], M, 10, 1 << 20, threads=8)
    assert np.array_equal(got["queries"].numpy()[idx].astype(np.int64), o["queries"])
    assert np.array_equal(got["cw"].numpy().view(np.uint32)[idx], o["cw"])
    code.close()


def test_caller_buffers_and_stream(g, oracle_lib):
    """Outputs into the caller's page-locked buffers; the caller's stream is
    ordered after the pipeline (an event recorded on it afterwards completes
    only after every chunk)."""
    import torch

    N, K, M = 512, 256, 64
    code = g.Code.polar(N, K)
    d = wl.qam_frames(3, 6, 3000, N, oracle_lib.info_set(N, K), M, 12.0)
    sym = torch.from_numpy(d["symbols"]).pin_memory()
    p = g.Params.make(M=M, S=12, query_cap=1 << 24)
    cw = torch.empty((3000, N // 32), dtype=torch.int32).pin_memory()
    q = torch.empty(3000, dtype=torch.int32).pin_memory()
    ab = torch.empty(3000, dtype=torch.uint8).pin_memory()
    s = torch.cuda.Stream()
    r = g.decode_symbols_host(code, p, sym, cw=cw, queries=q, abandon=ab, chunk_frames=1000, stream=s)
    assert r["cw"] is cw and r["queries"] is q and r["abandon"] is ab
    ev = torch.cuda.Event()
    ev.record(s)
    ev.synchronize()
    want = device_reference(g, code, p, sym)
    assert torch.equal(cw, want["cw"]) and torch.equal(q, want["queries"]) and torch.equal(ab, want["abandon"])
    code.close()


def test_bit_level_order(g, oracle_lib):
    import torch

    N, K = 32, 16
    code = g.Code.polar(N, K)
    d = wl.bpsk_frames(1, 3, 10000, N, oracle_lib.info_set(N, K), 4.0)
    sym = torch.from_numpy(d["symbols"]).pin_memory()
    p = g.Params.make(order=g.ORDER_HAMMING, M=2, S=0, max_weight=3, query_cap=5489)
    got = g.decode_symbols_host(code, p, sym, chunk_frames=3333)
    want = device_reference(g, code, p, sym)
    for k in ("cw", "queries", "abandon"):
        assert torch.equal(got[k], want[k]), k
    code.close()


def test_arguments(g):
    import torch

    code = g.Code.polar(128, 64)
    p = g.Params.make(M=16, S=10)
    empty = g.decode_symbols_host(code, p, torch.zeros((0, 32), dtype=torch.complex64))
    assert empty["queries"].numel() == 0
    with pytest.raises(g.GrandError) as e:  # checked before any device work
        g.decode_symbols_host(code, g.Params.make(M=16, S=-1), torch.zeros((4, 32), dtype=torch.complex64))
    assert e.value.status == -1
    with pytest.raises(g.GrandArgumentError):
        g.decode_symbols_host(code, p, torch.zeros((4, 32), dtype=torch.complex64, device="cuda"))
    with pytest.raises(g.GrandError):
        g.decode_symbols_host(code, p, torch.zeros((4, 32), dtype=torch.complex64), chunk_frames=-1)
    code.close()


def mixed_codes(g, oracle_lib, Ns):
    return [g.Code.polar(n, n // 2) for n in Ns]


def device_mixed(g, codes, p, desc, sym, n_cw):
    import torch

    r = g.decode_mixed(codes, p, torch.from_numpy(desc.view(np.uint8)).cuda(), sym.cuda(), n_cw)
    torch.cuda.synchronize()
    return {k: r[k].cpu() for k in ("cw", "queries", "abandon")}


@pytest.mark.parametrize("chunk", [7000, 0])
def test_mixed_equals_device_call(g, oracle_lib, chunk):
    """A packed uneven batch (every N and M) in chunks: same outputs as the
    device call."""
    import torch

    Ns = wl.MIXED_N
    codes = mixed_codes(g, oracle_lib, Ns)
    info = {n: oracle_lib.info_set(n, n // 2) for n in Ns}
    mx = wl.mixed_frames(9, 2, 30000, info)
    desc = g.frame_desc(np.searchsorted(np.array(Ns), mx["N"]), mx["M"], mx["sym_offset"], mx["cw_offset"])
    sym = torch.from_numpy(mx["symbols"]).pin_memory()
    p = g.Params.make(M=0, S=10, query_cap=1 << 20)
    want = device_mixed(g, codes, p, desc, sym, mx["n_cw_words"])
    got = g.decode_mixed_host(codes, p, desc, sym, mx["n_cw_words"], chunk_frames=chunk)
    for k in ("cw", "queries", "abandon"):
        assert torch.equal(got[k], want[k]), k
    for c in codes:
        c.close()


def test_mixed_unpacked_layout_and_bad_descriptor(g, oracle_lib):
    """Frames stored out of order with gaps between their output words: one
    chunk over the whole arrays; words no frame owns keep their values; a
    descriptor naming a missing code is reported with abandon 3."""
    import torch

    Ns = (64, 256)
    codes = mixed_codes(g, oracle_lib, Ns)
    rng = np.random.default_rng(3)
    parts, desc_rows, off = [], [], 0
    blocks = []
    for i, n in enumerate(Ns):
        d = wl.qam_frames(10, i, 200, n, oracle_lib.info_set(n, n // 2), 16, 6.0)
        blocks += [(i, 16, row) for row in d["symbols"]]
    order = rng.permutation(len(blocks))
    sym_parts, cw_off = [], 0
    for j, b in enumerate(order):
        ci, M, row = blocks[b]
        desc_rows.append((ci, M, off, cw_off))
        sym_parts.append(row)
        off += len(row)
        cw_off += Ns[ci] // 32 + 1  # one spare word after every frame
    desc_rows = desc_rows[::-1]  # descriptors in reverse storage order: not packed
    desc_rows[5] = (7, 16, desc_rows[5][2], desc_rows[5][3])  # no code 7
    desc = g.frame_desc(*map(np.array, zip(*desc_rows)))
    sym = torch.from_numpy(np.concatenate(sym_parts).astype(np.complex64)).pin_memory()
    p = g.Params.make(M=0, S=8, query_cap=1 << 16)
    cw = torch.full((cw_off,), 0x5A5A5A5A, dtype=torch.int32).pin_memory()
    got = g.decode_mixed_host(codes, p, desc, sym, cw_off, cw=cw, chunk_frames=50)
    want = device_mixed(g, codes, p, desc, sym, cw_off)
    assert torch.equal(got["queries"], want["queries"]) and torch.equal(got["abandon"], want["abandon"])
    assert int(got["abandon"][5]) == 3
    owned = np.zeros(cw_off, bool)
    for f, (ci, _, _, co) in enumerate(desc_rows):
        if f != 5:
            owned[co:co + Ns[ci] // 32] = True
    c = got["cw"].numpy()
    assert np.array_equal(c[owned], want["cw"].numpy()[owned])
    assert np.all(c[~owned] == 0x5A5A5A5A)
    for cd in codes:
        cd.close()
