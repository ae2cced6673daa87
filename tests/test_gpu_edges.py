"""GPU decoding of the hand-built edge cases of the oracle pins: equal keys
broken by symbol index, single and double symbol errors at the least reliable
ranks, and a hit exactly at the query cap (decoded) and one past it
(abandoned). Each case runs through the fused call and the two-call path and
must match the oracle and the value the pin derives by hand."""
from __future__ import annotations

import numpy as np
import pytest

import tests.test_oracle_pins as pins
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


def decode_both(g, code, sym, M, S, cap, order=1, membership=0):
    """Fused call and two-call path; they must agree. Returns (cw, queries, abandon)."""
    import torch

    d = torch.from_numpy(np.ascontiguousarray(sym)).cuda()
    p = g.Params.make(order=order, M=M, S=S, query_cap=cap, membership=membership)
    a = g.decode_symbols(code, p, d)
    dm = g.demod(d, M, code.N)
    b = g.decode_batch(code, p, dm["y"], dm["hard_idx"], dm["key"], dm["nmask"])
    torch.cuda.synchronize()
    for k in ("cw", "queries", "abandon"):
        assert torch.equal(a[k], b[k]), k
    return (a["cw"].cpu().numpy().view(np.uint32), a["queries"].cpu().numpy().astype(np.int64),
            a["abandon"].cpu().numpy())


@pytest.mark.parametrize("membership", [0, 3])
def test_equal_keys_break_by_index(g, oracle_lib, membership):
    """All 32 keys equal; symbol 3 sent at the neighbouring I point: query 11."""
    N, M = 128, 16
    code = g.Code.polar(N, 64)
    c = wl.random_codewords(wl.rng(8, 0), 1, N, oracle_lib.info_set(N, 64))
    d = oracle_lib.qam_d(M)
    tx = np.round(wl.qam_modulate(c, M)[0] / d)
    rx = tx - 0.25 * np.sign(tx.real) - 0.25j * np.sign(tx.imag)
    A = tx[3].real
    wrong = A - 2 * np.sign(A) if abs(A) == 3 else -A
    rx[3] = complex(wrong + 0.25 * np.sign(A), rx[3].imag)
    sym = (rx * d).astype(np.complex64)[None, :]
    cw, q, ab = decode_both(g, code, sym, M, 10, 1 << 20, membership=membership)
    assert (int(ab[0]), int(q[0])) == (0, 11)
    assert np.array_equal(cw[0], wl.pack_bits(c)[0])
    code.close()


def test_nearer_axis_and_five_point_single_errors(g, oracle_lib):
    """The two order-variant hand cases: query 3 / 2 (paper / nearer axis) for a
    vertical error, query 5 for an away-side error in the five-point order."""
    import torch

    N, M = 128, 16
    code = g.Code.polar(N, 64)
    c, s, i = pins._frame_with_moved_symbol(
        oracle_lib, lambda aI, aQ: True,
        lambda aI, aQ: complex(aI - 0.6 * np.sign(aI), aQ - 1.2 * np.sign(aQ)))
    _, q1, _ = decode_both(g, code, s, M, 8, 1 << 16, order=1)
    _, q2, _ = decode_both(g, code, s, M, 8, 1 << 16, order=2)
    assert (int(q1[0]), int(q2[0])) == (3, 2)
    c5, s5, _ = pins._frame_with_moved_symbol(
        oracle_lib, lambda aI, aQ: abs(aI) == 1 and abs(aQ) == 3,
        lambda aI, aQ: complex(aI - 0.5 * np.sign(aI), 0.7 * np.sign(aQ)))
    r = g.decode_symbols(code, g.Params.make(order=3, M=M, S=8, query_cap=1 << 16), torch.from_numpy(s5).cuda())
    torch.cuda.synchronize()
    assert int(r["abandon"][0]) == 0 and int(r["queries"][0]) == 5
    assert np.array_equal(r["cw"].cpu().numpy().view(np.uint32)[0], wl.pack_bits(c5)[0])
    code.close()


@pytest.mark.parametrize("membership", [0, 3])
def test_single_and_double_symbol_errors(g, oracle_lib, membership):
    """Codewords received near their points except one or two of the least
    reliable symbols, moved across a threshold: the search finds them, with
    the oracle's query counts."""
    N, M, S = 128, 16, 10
    code = g.Code.polar(N, 64)
    H = oracle_lib.parity_H(N, 64)
    info = oracle_lib.info_set(N, 64)
    gen = wl.rng(12, membership)
    c = wl.random_codewords(gen, 60, N, info)
    d = oracle_lib.qam_d(M)
    tx = np.round(wl.qam_modulate(c, M) / d)
    rx = tx + 0.05 * (gen.standard_normal(tx.shape) + 1j * gen.standard_normal(tx.shape))
    for f in range(60):
        for k, i in enumerate((5, 17)[: 1 + f % 2]):  # one error in even frames, two in odd ones
            A = tx[f, i].real
            toward = -np.sign(A)  # every 16-QAM level has a neighbour toward the centre
            rx[f, i] = complex(A + toward * (1.1 + 0.1 * k), rx[f, i].imag)
    sym = (rx * d).astype(np.complex64)
    want = oracle_lib.decode_qam(H, sym, M, S, 1 << 20)
    cw, q, ab = decode_both(g, code, sym, M, S, 1 << 20, membership=membership)
    assert np.array_equal(q, want["queries"]) and np.array_equal(ab, want["abandon"])
    assert np.array_equal(cw, want["cw"])
    assert np.all(ab == 0) and np.array_equal(cw, wl.pack_bits(c))
    code.close()


@pytest.mark.parametrize("membership", [0, 3])
def test_hit_exactly_at_the_cap(g, oracle_lib, membership):
    """A hit at query q decodes with cap q and abandons with cap q - 1
    (queries = q - 1, output = the hard word)."""
    N, M, S = 128, 16, 8
    code = g.Code.polar(N, 64)
    H = oracle_lib.parity_H(N, 64)
    dd = wl.qam_frames(4, 0, 200, N, oracle_lib.info_set(N, 64), M, 8.0)
    r = oracle_lib.decode_qam(H, dd["symbols"], M, S, 1 << 16)
    picks = np.nonzero((r["abandon"] == 0) & (r["queries"] > 50))[0][:6]
    assert picks.size >= 3
    for f in picks:
        qf = int(r["queries"][f])
        s = dd["symbols"][f:f + 1]
        cw, q, ab = decode_both(g, code, s, M, S, qf, membership=membership)
        assert (int(ab[0]), int(q[0])) == (0, qf) and np.array_equal(cw[0], r["cw"][f])
        cw, q, ab = decode_both(g, code, s, M, S, qf - 1, membership=membership)
        y = oracle_lib.demod(s, M, N)["y"][0]
        assert (int(ab[0]), int(q[0])) == (1, qf - 1) and np.array_equal(cw[0], y)
    code.close()
