"""The torch transmitter (used for the 10^6-frame BLER sweep) against the numpy
one: same codewords, same constellation points, same packing, for every
square QAM order; its noise has the channel's variance."""
from __future__ import annotations

import numpy as np
import pytest

import workloads as wl

torch = pytest.importorskip("torch")


@pytest.mark.parametrize("N,M", [(32, 4), (128, 16), (256, 64), (512, 256), (128, 1024), (64, 4096)])
def test_torch_transmitter_matches_numpy(oracle_lib, N, M):
    info = oracle_lib.info_set(N, N // 2)
    c = wl.random_codewords(wl.rng(99, N + M), 64, N, info)
    u = wl.polar_encode(c)  # the transform is an involution: these bits encode to c
    tx_t, c_t = wl.torch_encode_modulate(torch.from_numpy(u), M)
    assert np.array_equal(c_t.numpy(), c)
    assert np.array_equal(tx_t.numpy(), wl.qam_modulate(c, M))
    assert np.array_equal(wl.torch_pack_bits(c_t).numpy().view(np.uint32), wl.pack_bits(c))


def test_torch_frames_noise_and_codewords(oracle_lib):
    N, M, snr = 128, 16, 6.0
    info = oracle_lib.info_set(N, N // 2)
    d = wl.torch_qam_frames(7, 20000, N, info, M, snr, "cpu")
    H = oracle_lib.parity_H(N, N // 2)
    words = d["codewords_packed"].numpy().view(np.uint32)
    bits = ((words[:, :, None] >> np.arange(32, dtype=np.uint32)) & 1).reshape(len(words), N)
    assert not ((bits.astype(np.int64) @ H.T.astype(np.int64)) % 2).any()  # codewords
    tx, _ = wl.torch_encode_modulate(torch.from_numpy(wl.polar_encode(bits.astype(np.uint8))), M)
    noise = d["symbols"].numpy().astype(np.complex128) - tx.numpy()
    n0 = float(wl.ebn0_to_n0(snr))
    assert np.var(noise.real) == pytest.approx(n0 / 2, rel=0.02)
    assert np.var(noise.imag) == pytest.approx(n0 / 2, rel=0.02)
    assert abs(np.mean(noise.real)) < 0.01
    # the seed fixes the batch
    again = wl.torch_qam_frames(7, 20000, N, info, M, snr, "cpu")
    assert torch.equal(again["symbols"], d["symbols"])


def test_uneven_batch_is_packed_in_frame_order(oracle_lib):
    """The uneven-mix generator lays frames out back to back in frame order
    (each frame's symbols and output words right after the previous frame's),
    the layout the host-memory call cuts into chunks; the sent codewords sit at
    the output offsets and satisfy H c = 0."""
    info = {n: oracle_lib.info_set(n, n // 2) for n in wl.MIXED_N}
    mx = wl.mixed_frames(5, 3, 3000, info)
    L = np.array([wl.symbols_per_frame(int(n), int(m)) for n, m in zip(mx["N"], mx["M"])])
    assert np.array_equal(mx["L"], L)
    assert mx["sym_offset"][0] == 0 and mx["cw_offset"][0] == 0
    assert np.array_equal(np.diff(mx["sym_offset"]), L[:-1])
    assert np.array_equal(np.diff(mx["cw_offset"]), mx["N"][:-1] // 32)
    assert mx["n_sym"] == mx["sym_offset"][-1] + L[-1] == len(mx["symbols"])
    assert mx["n_cw_words"] == mx["cw_offset"][-1] + mx["N"][-1] // 32
    for f in range(0, 3000, 97):
        n, o = int(mx["N"][f]), int(mx["cw_offset"][f])
        words = mx["codewords_packed"][o:o + n // 32]
        bits = ((words[:, None] >> np.arange(32, dtype=np.uint32)) & 1).reshape(-1).astype(np.int64)
        H = oracle_lib.parity_H(n, n // 2).astype(np.int64)
        assert not (H @ bits % 2).any()
