"""Seeded synthetic inputs for the GRAND decoder: the transmitter and the channel.

This module is the only code shared by the CPU oracle side (tests, CPU baseline)
and the CUDA side (tests, benchmark). It holds no decoding arithmetic: it draws
information bits, encodes them with the polar transform c = u G_N (Def. II.1),
maps the coded bits to Gray-labelled square M-QAM points with spacing 2d
(Def. II.2, Eq. 2) or to BPSK, and adds white Gaussian noise (the AWGN channel
of Sec. IV). The code itself (which positions carry information) is an input.

Conventions (the paper's Fig. 1 is not in the text, so these are readings):
  * E_b = 1 per coded bit; N0 = 10^(-EbN0_dB/10); noise variance N0/2 per real
    dimension; d = sqrt(3 m E_b / (M - 1)) for M = 2^(2m) (Eq. 2).
  * L = ceil(N / 2m) symbols per codeword (Alg. 2 input); the coded word is
    padded with zero bits up to 2m L.
  * Symbol i carries bits [2m i, 2m i + 2m): the first m bits, most significant
    first, are the binary-reflected Gray label of the in-phase level, the next m
    bits that of the quadrature level. Level l in [0, 2^m) has odd-integer
    amplitude 2 l - (2^m - 1); its Gray label is l ^ (l >> 1).
  * BPSK: bit 0 -> +1, bit 1 -> -1.
  * Noise is drawn in float64 from numpy's Philox generator, added in float64,
    and the received values are rounded once to complex64 / float32.
"""
from __future__ import annotations

import math

import numpy as np

SEED_BASE = 0x240501808

QAM_ORDERS = (4, 16, 64, 256)


def rng(config_id: int, stream: int = 0) -> np.random.Generator:
    """Counter-based generator for one (config, stream) pair (Philox4x32-10)."""
    key = (SEED_BASE ^ (int(config_id) * 0x9E3779B97F4A7C15)) & ((1 << 64) - 1)
    return np.random.Generator(np.random.Philox(key=[key, int(stream)]))


def bits_per_symbol(M: int) -> int:
    b = int(round(math.log2(M)))
    if M < 4 or (1 << b) != M or b % 2:
        raise ValueError(f"M={M} is not a square QAM order 2^(2m)")
    return b


def symbols_per_frame(N: int, M: int) -> int:
    """L = ceil(N / log2 M) (Alg. 2 input)."""
    return -(-N // bits_per_symbol(M))


def ebn0_to_n0(ebn0_db: float | np.ndarray) -> np.ndarray:
    return np.power(10.0, -np.asarray(ebn0_db, dtype=np.float64) / 10.0)


def polar_encode(u: np.ndarray) -> np.ndarray:
    """c = u G_N with G_N = F^{(x)n}, F = [[1,0],[1,1]], over GF(2) (Def. II.1).

    u: uint8 array (..., N) of 0/1. Implemented as n butterfly stages: entry
    G[i][j] is 1 exactly when the bit set of j is contained in that of i, so
    c_j is the XOR of u_i over all i that contain j.
    """
    c = np.array(u, dtype=np.uint8, copy=True)
    N = c.shape[-1]
    lead = c.shape[:-1]
    half = 1
    while half < N:
        v = c.reshape(lead + (N // (2 * half), 2, half))
        v[..., 0, :] ^= v[..., 1, :]
        half *= 2
    return c


def pack_bits(bits: np.ndarray) -> np.ndarray:
    """(F, N) 0/1 -> (F, ceil(N/32)) uint32, bit j at word j>>5, bit j&31."""
    F, N = bits.shape
    W = -(-N // 32)
    padded = np.zeros((F, W * 32), dtype=np.uint64)
    padded[:, :N] = bits
    shifts = np.arange(32, dtype=np.uint64)
    words = (padded.reshape(F, W, 32) << shifts).sum(axis=2)
    return words.astype(np.uint32)


def random_codewords(g: np.random.Generator, n_frames: int, N: int, info_positions) -> np.ndarray:
    """Uniform information bits on `info_positions`, zeros elsewhere, encoded."""
    info = np.asarray(info_positions, dtype=np.int64)
    u = np.zeros((n_frames, N), dtype=np.uint8)
    u[:, info] = g.integers(0, 2, size=(n_frames, info.size), dtype=np.uint8)
    return polar_encode(u)


def qam_modulate(codewords: np.ndarray, M: int) -> np.ndarray:
    """Coded bits (F, N) -> transmitted points (F, L) complex128 in units of E_b = 1."""
    b = bits_per_symbol(M)
    m = b // 2
    F, N = codewords.shape
    L = -(-N // b)
    bits = np.zeros((F, L * b), dtype=np.int64)
    bits[:, :N] = codewords
    bits = bits.reshape(F, L, b)
    weights = 1 << np.arange(m - 1, -1, -1, dtype=np.int64)  # MSB first
    gI = (bits[:, :, :m] * weights).sum(axis=2)
    gQ = (bits[:, :, m:] * weights).sum(axis=2)
    side = 1 << m
    # inverse of the Gray map g = l ^ (l >> 1)
    gray = np.arange(side) ^ (np.arange(side) >> 1)
    level_of = np.empty(side, dtype=np.int64)
    level_of[gray] = np.arange(side)
    aI = 2 * level_of[gI] - (side - 1)
    aQ = 2 * level_of[gQ] - (side - 1)
    d = math.sqrt(3.0 * m / (M - 1))
    return d * (aI + 1j * aQ)


def awgn(g: np.random.Generator, tx: np.ndarray, n0: np.ndarray | float) -> np.ndarray:
    """Add complex (or real) Gaussian noise with variance N0/2 per dimension."""
    n0 = np.asarray(n0, dtype=np.float64)
    sigma = np.sqrt(n0 / 2.0)
    if n0.ndim == 1:
        sigma = sigma.reshape((-1,) + (1,) * (tx.ndim - 1))
    if np.iscomplexobj(tx):
        noise = g.standard_normal(tx.shape + (2,))
        return tx + sigma * (noise[..., 0] + 1j * noise[..., 1])
    return tx + sigma * g.standard_normal(tx.shape)


def qam_frames(config_id: int, stream: int, n_frames: int, N: int, info_positions, M: int,
               ebn0_db: float) -> dict:
    """One uniform batch: received complex64 symbols (F, L) and the sent codewords."""
    g = rng(config_id, stream)
    c = random_codewords(g, n_frames, N, info_positions)
    tx = qam_modulate(c, M)
    rx = awgn(g, tx, float(ebn0_to_n0(ebn0_db)))
    return {
        "symbols": rx.astype(np.complex64),
        "codewords": c,
        "codewords_packed": pack_bits(c),
        "N": N, "M": M, "L": tx.shape[1], "ebn0_db": float(ebn0_db),
        "n0": float(ebn0_to_n0(ebn0_db)),
    }


def bpsk_frames(config_id: int, stream: int, n_frames: int, N: int, info_positions,
                ebn0_db: float) -> dict:
    g = rng(config_id, stream)
    c = random_codewords(g, n_frames, N, info_positions)
    tx = 1.0 - 2.0 * c.astype(np.float64)
    rx = awgn(g, tx, float(ebn0_to_n0(ebn0_db)))
    return {
        "symbols": rx.astype(np.float32),
        "codewords": c,
        "codewords_packed": pack_bits(c),
        "N": N, "M": 2, "L": N, "ebn0_db": float(ebn0_db),
        "n0": float(ebn0_to_n0(ebn0_db)),
    }


MIXED_N = (32, 64, 128, 256, 512, 1024)


def mixed_frames(config_id: int, stream: int, n_frames: int, info_by_N: dict,
                 ebn0_range=(4.0, 14.0), n_choices=MIXED_N, m_choices=QAM_ORDERS) -> dict:
    """Uneven batch: per frame N, M and E_b/N0 drawn uniformly; symbols concatenated.

    Returns flat complex64 `symbols`, per-frame `N`, `M`, `L`, `sym_offset`
    (in symbols), `cw_offset` (in 32-bit words), `ebn0_db`, and the sent
    codewords packed into a flat uint32 array at `cw_offset`.
    """
    g = rng(config_id, stream)
    Ns = g.choice(np.asarray(n_choices, dtype=np.int64), size=n_frames)
    Ms = g.choice(np.asarray(m_choices, dtype=np.int64), size=n_frames)
    snr = g.uniform(ebn0_range[0], ebn0_range[1], size=n_frames)
    Ls = np.array([symbols_per_frame(int(n), int(m)) for n, m in zip(Ns, Ms)], dtype=np.int64)
    sym_off = np.zeros(n_frames + 1, dtype=np.int64)
    np.cumsum(Ls, out=sym_off[1:])
    cw_words = Ns // 32
    cw_off = np.zeros(n_frames + 1, dtype=np.int64)
    np.cumsum(cw_words, out=cw_off[1:])
    symbols = np.empty(int(sym_off[-1]), dtype=np.complex64)
    cw_packed = np.empty(int(cw_off[-1]), dtype=np.uint32)
    for n in np.unique(Ns):
        for m in np.unique(Ms):
            idx = np.nonzero((Ns == n) & (Ms == m))[0]
            if idx.size == 0:
                continue
            c = random_codewords(g, idx.size, int(n), info_by_N[int(n)])
            tx = qam_modulate(c, int(m))
            rx = awgn(g, tx, ebn0_to_n0(snr[idx])).astype(np.complex64)
            L = tx.shape[1]
            pos = sym_off[idx][:, None] + np.arange(L)[None, :]
            symbols[pos.ravel()] = rx.ravel()
            W = int(n) // 32
            wpos = cw_off[idx][:, None] + np.arange(W)[None, :]
            cw_packed[wpos.ravel()] = pack_bits(c).ravel()
    return {
        "symbols": symbols, "N": Ns.astype(np.int32), "M": Ms.astype(np.int32),
        "L": Ls.astype(np.int32), "sym_offset": sym_off[:-1].copy(), "cw_offset": cw_off[:-1].copy(),
        "ebn0_db": snr, "codewords_packed": cw_packed, "n_sym": int(sym_off[-1]),
        "n_cw_words": int(cw_off[-1]),
    }


# ---------------------------------------------------------------------------
# The same transmitter and channel in torch, on any device, for sweeps whose
# frame counts make host generation the bottleneck (10^6 frames per point).
# It follows the conventions above step by step; the noise comes from a
# seeded torch generator (not numpy's Philox stream), so its draws differ
# from qam_frames for the same seed while the distribution is the same.
# ---------------------------------------------------------------------------
def torch_encode_modulate(u, M: int):
    """Information-position bits u (F, N) uint8 tensor -> (tx complex128 (F, L),
    codeword bits (F, N) uint8): polar transform, padding, Gray QAM map."""
    import torch

    c = u.clone()
    F, N = c.shape
    half = 1
    while half < N:
        v = c.view(F, N // (2 * half), 2, half)
        v[:, :, 0, :] ^= v[:, :, 1, :]
        half *= 2
    b = bits_per_symbol(M)
    m = b // 2
    L = -(-N // b)
    bits = torch.zeros((F, L * b), dtype=torch.int32, device=c.device)
    bits[:, :N] = c.to(torch.int32)
    bits = bits.view(F, L, b)
    weights = (1 << torch.arange(m - 1, -1, -1, device=c.device, dtype=torch.int32))
    gI = (bits[:, :, :m] * weights).sum(dim=2)
    gQ = (bits[:, :, m:] * weights).sum(dim=2)
    side = 1 << m
    levels = torch.arange(side, device=c.device, dtype=torch.int64)
    level_of = torch.empty(side, dtype=torch.int64, device=c.device)
    level_of[levels ^ (levels >> 1)] = levels
    aI = (2 * level_of[gI.long()] - (side - 1)).to(torch.float64)
    aQ = (2 * level_of[gQ.long()] - (side - 1)).to(torch.float64)
    d = math.sqrt(3.0 * m / (M - 1))
    return torch.complex(d * aI, d * aQ), c


def torch_pack_bits(bits):
    """(F, N) 0/1 tensor, N a multiple of 32 -> (F, N/32) int32 words (bit j at word j>>5, bit j&31)."""
    import torch

    F, N = bits.shape
    w = bits.to(torch.int64).view(F, N // 32, 32) << torch.arange(32, device=bits.device, dtype=torch.int64)
    return ((w.sum(dim=2) + (1 << 31)) % (1 << 32) - (1 << 31)).to(torch.int32)  # two's complement


def torch_qam_frames(seed: int, n_frames: int, N: int, info_positions, M: int, ebn0_db: float, device):
    """A uniform batch generated on `device`: received complex64 symbols (F, L)
    and the sent codewords packed (F, N/32) int32."""
    import torch

    gen = torch.Generator(device=device)
    gen.manual_seed(int(seed))
    info = torch.as_tensor(np.asarray(info_positions, dtype=np.int64), device=device)
    u = torch.zeros((n_frames, N), dtype=torch.uint8, device=device)
    u[:, info] = torch.randint(0, 2, (n_frames, info.numel()), generator=gen, device=device, dtype=torch.uint8)
    tx, c = torch_encode_modulate(u, M)
    sigma = math.sqrt(float(ebn0_to_n0(ebn0_db)) / 2.0)
    noise = torch.randn(tx.shape + (2,), generator=gen, device=device, dtype=torch.float64) * sigma
    rx = torch.complex(tx.real + noise[..., 0], tx.imag + noise[..., 1]).to(torch.complex64)
    return {"symbols": rx, "codewords_packed": torch_pack_bits(c)}
