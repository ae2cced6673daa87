"""Theorem III.1 and Table II (Sec. III): the printed table is checked for
internal consistency, and the theorem's step count is recomputed on this
project's parity-check matrices by an explicit pairwise XOR tree per row (the
shape of Alg. 1's product), whose result must equal the direct GF(2) product.
The paper's H basis differs from this project's (its frozen set and null-space
basis are not in the text), so its numbers are not compared with ours. CPU only."""
from __future__ import annotations

import math
import os

import numpy as np
import pytest

import workloads as wl

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "table2_summary.txt")


def _rows():
    out = []
    for line in open(GOLDEN):
        line = line.strip()
        if line and not line.startswith("#"):
            n, N, wh, sp, mx, xor, cc = line.split()
            out.append((int(n), int(N), int(wh), float(sp), int(mx), int(xor), int(cc)))
    return out


def test_table2_internal_consistency():
    rows = _rows()
    assert [r[0] for r in rows] == list(range(5, 11))
    for n, N, wh, sp, mx, xor, cc in rows:
        assert N == 2 ** n
        K = N // 2
        assert round(100.0 * wh / (K * N), 2) == pytest.approx(sp, abs=0.006)  # sparsity = W_H / (K N)
        assert cc == 1 + math.ceil(math.log2(mx))                                # Thm. III.1 step count
        assert cc <= n                                                           # bounded by log2 N (Prop. III.1)
        assert mx <= N and wh <= K * N and xor < wh
    wh7, xor7 = rows[2][2], rows[2][5]
    assert wh7 * 2 ** 16 == pytest.approx(64.5e6, rel=0.01)  # AND gates for 2^16 instances at n = 7
    assert xor7 * 2 ** 16 == pytest.approx(16.2e6, rel=0.01)  # XOR gates likewise


def _xor_tree(bits):
    """Pairwise XOR reduction of the row's products (one level per step);
    returns (parity, levels)."""
    level = list(bits)
    depth = 0
    while len(level) > 1:
        nxt = [level[i] ^ level[i + 1] for i in range(0, len(level) - 1, 2)]
        if len(level) % 2:
            nxt.append(level[-1])  # the odd element moves up unchanged
        level = nxt
        depth += 1
    return (level[0] if level else 0), depth


@pytest.mark.parametrize("N", [32, 64, 128])
def test_theorem_iii1_on_this_projects_H(oracle_lib, N):
    K = N // 2
    H = oracle_lib.parity_H(N, K).astype(np.int64)
    weights = H.sum(axis=1)
    steps = 1 + max(math.ceil(math.log2(w)) for w in weights)   # Thm. III.1
    g = np.random.default_rng(N)
    info = oracle_lib.info_set(N, K)
    words = np.concatenate([g.integers(0, 2, size=(20, N)), wl.random_codewords(wl.rng(98, N), 20, N, info)])
    seen_depth = 0
    for c in words:
        for r in range(N - K):
            ones = np.nonzero(H[r])[0]
            parity, depth = _xor_tree([int(c[j]) for j in ones])   # AND step, then the tree
            assert parity == int(H[r] @ c) % 2
            assert depth == math.ceil(math.log2(len(ones)))
            seen_depth = max(seen_depth, depth)
    assert 1 + seen_depth == steps
    # this H: rows are columns of G_N at the frozen indices, weight 2^(n - popcount(f));
    # the all-ones row (frozen index 0) makes the step count n + 1, one above the
    # paper's bound for its own basis
    n = int(math.log2(N))
    f = oracle_lib.frozen_set(N, K)
    assert np.array_equal(np.sort(weights), np.sort([2 ** (n - bin(int(x)).count("1")) for x in f]))
    assert steps == n + 1
