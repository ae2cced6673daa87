"""The binding's argument checks (no GPU needed: they run before any library
call and before the device check). The library takes bare pointers and trusts
their sizes, so every tensor's element type and count is checked against what
the call reads or writes."""
from __future__ import annotations

import types

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import paper_2405_01808_gb300 as g  # noqa: E402

CODE = types.SimpleNamespace(N=128, K=64, handle=None)  # stands in for a code object


def expect(fragment, fn, *args, **kw):
    with pytest.raises(g.GrandArgumentError) as e:
        fn(*args, **kw)
    assert fragment in str(e.value), str(e.value)
    assert e.value.status == -1 and isinstance(e.value, ValueError) and isinstance(e.value, g.GrandError)


def test_symbols_type_and_shape():
    p = g.Params.make(M=16, S=10)
    expect("dtype", g.decode_symbols, CODE, p, torch.zeros((4, 32), dtype=torch.complex128))
    expect("exactly 128", g.decode_symbols, CODE, p, torch.zeros((4, 31), dtype=torch.complex64))
    expect("exactly 256", g.decode_symbols, CODE, p, torch.zeros((4, 32, 1), dtype=torch.float32))
    # the right type and size on the host: only the device is wrong
    expect("CUDA device", g.decode_symbols, CODE, p, torch.zeros((4, 32), dtype=torch.complex64))
    expect("CUDA device", g.decode_symbols, CODE, p, torch.zeros((4, 32, 2), dtype=torch.float32))
    # 64-QAM: L = ceil(128 / 6) = 22
    expect("exactly 88", g.decode_symbols, CODE, g.Params.make(M=64, S=10), torch.zeros((4, 32), dtype=torch.complex64))
    expect("square constellation", g.decode_symbols, CODE, g.Params.make(M=8, S=10),
           torch.zeros((4, 32), dtype=torch.complex64))


def test_bpsk_samples():
    p = g.Params.make(order=g.ORDER_HAMMING, M=2, S=0, max_weight=3, query_cap=5489)
    expect("exactly 512", g.decode_symbols, CODE, p, torch.zeros((4, 64), dtype=torch.float32))
    expect("dtype", g.decode_symbols, CODE, p, torch.zeros((4, 128), dtype=torch.float64))
    expect("CUDA device", g.decode_symbols, CODE, p, torch.zeros((4, 128), dtype=torch.float32))


def test_output_buffers():
    p = g.Params.make(M=16, S=10)
    x = torch.zeros((4, 32), dtype=torch.complex64)
    expect("cw", g.decode_symbols, CODE, p, x, cw=torch.zeros(15, dtype=torch.int32))
    expect("queries: dtype", g.decode_symbols, CODE, p, x, queries=torch.zeros(4, dtype=torch.int64))
    expect("abandon", g.decode_symbols, CODE, p, x, abandon=torch.zeros(3, dtype=torch.uint8))
    ok = dict(cw=torch.zeros((4, 4), dtype=torch.int32), queries=torch.zeros(4, dtype=torch.int32),
              abandon=torch.zeros(4, dtype=torch.uint8))
    expect("CUDA device", g.decode_symbols, CODE, p, x, **ok)
    expect("cw is required", g.decode_symbols_noalloc, CODE, p, x, None, ok["queries"], ok["abandon"])


def test_demodulated_inputs():
    p = g.Params.make(M=16, S=10)
    y = torch.zeros((4, 4), dtype=torch.int32)
    hi = torch.zeros((4, 32), dtype=torch.int16)
    key = torch.zeros((4, 32), dtype=torch.int32)
    nm = torch.zeros((4, 32), dtype=torch.uint8)
    expect("key is required", g.decode_batch, CODE, p, y, hi, None, nm)
    expect("hard_idx", g.decode_batch, CODE, p, y, hi[:, :16].contiguous(), key, nm)
    expect("key: dtype", g.decode_batch, CODE, p, y, hi, key.float(), nm)
    expect("y: 12 elements", g.decode_batch, CODE, p, y[:, :3].contiguous(), hi, key, nm)
    expect("CUDA device", g.decode_batch, CODE, p, y, hi, key, nm)


def test_demod_outputs():
    x = torch.zeros((4, 32), dtype=torch.complex64)
    expect("square constellation", g.demod, x, 8, 128)
    expect("exactly 88", g.demod, x, 64, 128)
    expect("CUDA device", g.demod, x, 16, 128)


def test_mixed_batch_records():
    desc = torch.from_numpy(g.frame_desc([0, 0], [16, 16], [0, 32], [0, 4]).view(np.uint8))
    sym = torch.zeros(64, dtype=torch.complex64)
    expect("whole number", g.decode_mixed, [CODE], g.Params.make(M=0, S=10), desc[:-1].contiguous(), sym, 8)
    expect("float32 pairs", g.decode_mixed, [CODE], g.Params.make(M=0, S=10), desc, torch.zeros(7), 8)
    expect("cw", g.decode_mixed, [CODE], g.Params.make(M=0, S=10), desc, sym, 8,
           cw=torch.zeros(7, dtype=torch.int32))
    expect("CUDA device", g.decode_mixed, [CODE], g.Params.make(M=0, S=10), desc, sym, 8)


def test_host_memory_call():
    p = g.Params.make(M=16, S=10)
    expect("exactly 128", g.decode_symbols_host, CODE, p, torch.zeros((4, 31), dtype=torch.complex64))
    expect("queries: dtype", g.decode_symbols_host, CODE, p, torch.zeros((4, 32), dtype=torch.complex64),
           queries=torch.zeros(4, dtype=torch.int64))


def test_mixed_host_memory_call():
    desc = g.frame_desc([0, 0], [16, 16], [0, 32], [0, 4])
    p = g.Params.make(M=0, S=10)
    expect("whole number", g.decode_mixed_host, [CODE], p, torch.from_numpy(desc.view(np.uint8))[:-1].contiguous(),
           torch.zeros(64, dtype=torch.complex64), 8)
    expect("dtype", g.decode_mixed_host, [CODE], p, desc, torch.zeros(64, dtype=torch.complex128), 8)
    expect("cw", g.decode_mixed_host, [CODE], p, desc, torch.zeros(64, dtype=torch.complex64), 8,
           cw=torch.zeros(7, dtype=torch.int32))
