"""The stored full-size expected outputs (tests/golden/fullsize_*.npz) are the
oracle's: each file's invariants hold (shapes, flags, abandoned frames keep
their hard word, queries within the cap), a sample of its frames, re-decoded
here by the oracle, comes out identical, and a sample of its abandoned frames
abandons under the oracle at a short cap too. The GPU path never writes these files;
tests/golden/make_fullsize_golden.py does, from the oracle and the input
generator alone. Run on the CPU."""
from __future__ import annotations

import hashlib
import json
import os

import numpy as np
import pytest

import workloads as wl

GOLDEN = os.path.dirname(os.path.abspath(__file__)) + "/golden"
CONFIGS = {
    "c2": dict(cid=2, N=128, M=16, snrs=(6.0, 8.0, 10.0), frames=100000),
    "c3a": dict(cid=3, N=512, M=64, snrs=(10.0, 12.0, 14.0, 16.0), frames=20000),
    "c3b": dict(cid=4, N=1024, M=256, snrs=(10.0, 12.0, 14.0, 16.0), frames=20000),
}


def load(config):
    path = os.path.join(GOLDEN, f"fullsize_{config}.npz")
    assert os.path.exists(path), f"missing {path}"
    z = np.load(path, allow_pickle=False)
    return z, json.loads(str(z["meta"]))


@pytest.mark.parametrize("config", ["c2", "c3a", "c3b", "c4"])
def test_golden_invariants(config):
    z, meta = load(config)
    assert meta["config"] == config and meta["strata"]
    expect = {"c2": 3, "c3a": 4, "c3b": 4, "c4": 24}[config]
    assert len(meta["strata"]) == expect
    for name, st in meta["strata"].items():
        n = int(st["n"])
        q, ab, e = z[f"{name}_queries"], z[f"{name}_abandon"], z[f"{name}_e"]
        assert q.shape == (n,) and ab.shape == (n,) and e.shape == (n, st["N"] // 32)
        assert set(np.unique(ab).tolist()) <= {0, 1}
        assert np.all(q >= 1) and np.all(q.astype(np.int64) <= st["cap"])
        assert not e[ab == 1].any(), "an abandoned frame keeps its hard word"
        assert np.all(q[ab == 0] > 0)
        # a decoded frame at query 1 is its hard word (t = 0 is the empty TEP)
        assert not e[(ab == 0) & (q == 1)].any()
        assert int((ab == 1).sum()) == st["abandons"]
        if config == "c2":
            assert n == st["frames_in_batch"] == 100000


def _sample(q, ab, cap_q, k, rng):
    """Up to k frames whose oracle decode is cheap (queries <= cap_q), plus
    the decoded frame with the most queries under that bound."""
    cheap = np.nonzero(q.astype(np.int64) <= cap_q)[0]
    if cheap.size == 0:
        return cheap
    pick = rng.choice(cheap, size=min(k, cheap.size), replace=False)
    dec = cheap[ab[cheap] == 0]
    if dec.size:
        pick = np.append(pick, dec[np.argmax(q[dec])])
    return np.unique(pick)


def _check_abandons(oracle_lib, H, sym, M, S, q, ab, rng, k=4, short_cap=2000):
    """A stored abandon says no codeword among the frame's first `cap` valid
    TEPs, so there is none among its first short_cap either: the oracle at
    that cap must abandon too, after min(short_cap, stored count) queries."""
    idx = np.nonzero(ab == 1)[0]
    if idx.size == 0:
        return 0
    idx = np.sort(rng.choice(idx, size=min(k, idx.size), replace=False))
    want = oracle_lib.decode_qam(H, sym[idx], M, S, short_cap, threads=os.cpu_count() or 1)
    assert np.all(want["abandon"] == 1)
    assert np.array_equal(want["queries"], np.minimum(short_cap, q[idx].astype(np.int64)))
    return idx.size


@pytest.mark.parametrize("config", ["c2", "c3a", "c3b"])
def test_golden_sample_equals_oracle(oracle_lib, config):
    """Re-decode a sample of each SNR stratum with the oracle (frames whose
    search is short enough for a CPU test) and compare with the file; check
    a sample of its abandoned frames at a short cap."""
    z, meta = load(config)
    c = CONFIGS[config]
    N, M = c["N"], c["M"]
    info = oracle_lib.info_set(N, N // 2)
    H = oracle_lib.parity_H(N, N // 2)
    rng = np.random.default_rng(11)
    for i, snr in enumerate(c["snrs"]):
        name = f"s{i}"
        st = meta["strata"][name]
        n = int(st["n"])
        # the stratum is a prefix of the whole SNR batch (whose draws depend on its size)
        sym = wl.qam_frames(c["cid"], i, c["frames"], N, info, M, snr)["symbols"][:n]
        assert hashlib.sha256(np.ascontiguousarray(sym, dtype=np.complex64).tobytes()).hexdigest() == \
            st["symbols_sha256"]
        q, ab, e = z[f"{name}_queries"], z[f"{name}_abandon"], z[f"{name}_e"]
        checked = _check_abandons(oracle_lib, H, sym, M, st["S"], q, ab, rng)
        idx = _sample(q, ab, 20000 if N == 128 else 3000, 12, rng)
        assert idx.size + checked > 0
        if idx.size == 0:
            continue  # every stored frame of the stratum abandons at the cap
        want = oracle_lib.decode_qam(H, sym[idx], M, st["S"], st["cap"], threads=os.cpu_count() or 1)
        y = oracle_lib.demod(sym[idx], M, N)["y"]
        assert np.array_equal(want["queries"], q[idx].astype(np.int64))
        assert np.array_equal(want["abandon"], ab[idx])
        assert np.array_equal(want["cw"], y ^ e[idx])


def test_golden_mix_sample_equals_oracle(oracle_lib):
    z, meta = load("c4")
    info = {n: oracle_lib.info_set(n, n // 2) for n in wl.MIXED_N}
    mx = wl.mixed_frames(5, 1000, 1000000, info)
    rng = np.random.default_rng(12)
    for n in (32, 128, 512):
        H = oracle_lib.parity_H(n, n // 2)
        for M in (4, 64):
            name = f"n{n}_m{M}"
            st = meta["strata"][name]
            f = np.nonzero((mx["N"] == n) & (mx["M"] == M))[0][: int(st["n"])]
            L = wl.symbols_per_frame(n, M)
            sym = mx["symbols"][mx["sym_offset"][f][:, None] + np.arange(L)[None, :]]
            q, ab, e = z[f"{name}_queries"], z[f"{name}_abandon"], z[f"{name}_e"]
            _check_abandons(oracle_lib, H, sym, M, st["S"], q, ab, rng, k=2)
            idx = _sample(q, ab, 5000, 8, rng)
            want = oracle_lib.decode_qam(H, sym[idx], M, st["S"], st["cap"], threads=os.cpu_count() or 1)
            y = oracle_lib.demod(sym[idx], M, n)["y"]
            assert np.array_equal(want["queries"], q[idx].astype(np.int64)), name
            assert np.array_equal(want["abandon"], ab[idx]), name
            assert np.array_equal(want["cw"], y ^ e[idx]), name
