"""The reading behind GRAND_MEMBERSHIP_SOLVE, pinned on the CPU against the
oracle's canonical TEP order (no GPU code involved).

Over the S' ranks every rank offers the alternatives that exist among h, v
and the diagonal (Def. III.2), and the diagonal exists exactly when h and v
do, so the valid TEPs are the flip vectors x over the existing I / Q slots.
The syndrome of y xor e(x) is s(y) xor (XOR of the slot columns over x), so
the codewords of the TEP space are the solutions of a GF(2) linear system,
and Alg. 2 Step 5's first hit is the solution of smallest canonical rank.
These tests build small instances (H of a polar code, slot positions with
repeated columns, padding slots and dependent sets, existence patterns,
syndromes inside and outside the slot span), walk the oracle's canonical
order until the first zero syndrome, and compare with an elimination written
here from that reading."""
from __future__ import annotations

import numpy as np
import pytest

NO_POS = -1  # a flip beyond N (padding bits): the slot exists, its column is zero


def columns(H, pos):
    """Syndrome column of every slot (2 per rank); zero for NO_POS."""
    R = H.shape[0]
    return np.stack([H[:, p] if p != NO_POS else np.zeros(R, np.uint8) for p in pos], axis=1)


def first_hit_by_walk(oracle_lib, cols, s0, exists):
    """Alg. 2 Step 5 as written: valid TEPs in canonical order, first zero syndrome."""
    codes, total = oracle_lib.tep_order(exists, max_out=1 << 18)
    assert len(codes) == total
    for i, c in enumerate(codes):
        z = s0.copy()
        for b in range(2 * len(exists)):
            if (int(c) >> b) & 1:
                z ^= cols[:, b]
        if not z.any():
            return i + 1, int(c), total
    return None, None, total


def first_hit_by_solve(oracle_lib, cols, s0, exists):
    """The reading: Gaussian elimination over the existing slots; the
    solutions x0 + span(kernel); the first hit is the one of smallest rank."""
    n = cols.shape[1]
    on = [b for b in range(n) if (exists[b >> 1] >> (b & 1)) & 1]
    # augmented columns with the set of original slots each one sums
    work = [(cols[:, b].copy(), 1 << b) for b in on]
    rhs, rmask = s0.copy(), 0
    basis = []  # (pivot row, column, mask)
    kernel = []
    for v, m in work:
        for prow, pv, pm in basis:
            if v[prow]:
                v ^= pv
                m ^= pm
        nz = np.nonzero(v)[0]
        if nz.size == 0:
            kernel.append(m)
            continue
        basis.append((int(nz[0]), v, m))
    for prow, pv, pm in basis:
        if rhs[prow]:
            rhs ^= pv
            rmask ^= pm
    codes, total = oracle_lib.tep_order(exists, max_out=1 << 18)
    rank_of = {int(c): i + 1 for i, c in enumerate(codes)}
    if rhs.any():
        return None, None, total
    best = None
    for sel in range(1 << len(kernel)):
        x = rmask
        for t, k in enumerate(kernel):
            if (sel >> t) & 1:
                x ^= k
        r = rank_of[x]  # every solution is a valid TEP
        if best is None or r < best[0]:
            best = (r, x)
    return best[0], best[1], total


def random_instance(rng, H, Sp, with_solution, pad_share=0.1, dependent=False):
    R, N = H.shape
    pos = [int(p) for p in rng.choice(N, size=2 * Sp, replace=False)]
    if dependent and Sp >= 2:
        pos[3] = pos[0]  # two slots flip the same bit: equal columns
    for b in range(2 * Sp):
        if rng.random() < pad_share:
            pos[b] = NO_POS
    exists = rng.choice(np.array([7, 7, 7, 1, 2, 0], np.uint8), size=Sp)
    cols = columns(H, pos)
    if with_solution:
        x = 0
        for b in range(2 * Sp):
            if (exists[b >> 1] >> (b & 1)) & 1 and rng.random() < 0.3:
                x |= 1 << b
        s0 = np.zeros(R, np.uint8)
        for b in range(2 * Sp):
            if (x >> b) & 1:
                s0 ^= cols[:, b]
    else:
        s0 = rng.integers(0, 2, size=R).astype(np.uint8)
    return cols, s0, exists


@pytest.mark.parametrize("N,K", [(32, 16), (64, 32), (128, 64)])
def test_first_hit_is_the_smallest_ranked_solution(oracle_lib, N, K):
    H = oracle_lib.parity_H(N, K)
    rng = np.random.default_rng(2405 + N)
    seen = {"hit": 0, "none": 0, "kernel": 0}
    for trial in range(60):
        Sp = int(rng.integers(1, 8))
        cols, s0, exists = random_instance(rng, H, Sp, with_solution=trial % 3 != 0,
                                           dependent=trial % 5 == 0)
        want = first_hit_by_walk(oracle_lib, cols, s0, exists)
        got = first_hit_by_solve(oracle_lib, cols, s0, exists)
        assert got == want, (N, trial, Sp, exists.tolist())
        seen["hit" if want[0] else "none"] += 1
    assert seen["hit"] > 20 and seen["none"] > 5


def test_dependent_slots_pick_the_earliest_solution(oracle_lib):
    """A set of slot columns that sums to zero (the support of a low-weight
    codeword, or two slots on one bit) gives several solutions; the first
    hit is the earliest of them in canonical order, not the eliminations' x0."""
    N, K = 32, 16
    H = oracle_lib.parity_H(N, K)
    # a codeword of the code: its support's columns sum to zero
    G = oracle_lib.generator_G(N)
    info = oracle_lib.info_set(N, K)
    u = np.zeros(N, np.uint8)
    u[info[-1]] = 1
    c = (u @ G) % 2
    supp = [int(j) for j in np.nonzero(c)[0]]
    assert not ((H.astype(np.int64) @ c) % 2).any()
    rng = np.random.default_rng(7)
    multi = 0
    for trial in range(40):
        Sp = max(4, (len(supp) + 1) // 2)
        Sp = min(Sp, 7)
        pos = list(supp[: 2 * Sp]) + [int(p) for p in rng.choice(N, size=2 * Sp, replace=False)]
        pos = pos[: 2 * Sp]
        exists = np.full(Sp, 7, np.uint8)
        cols = columns(H, pos)
        x = int(rng.integers(0, 1 << (2 * Sp)))
        s0 = np.zeros(H.shape[0], np.uint8)
        for b in range(2 * Sp):
            if (x >> b) & 1:
                s0 ^= cols[:, b]
        want = first_hit_by_walk(oracle_lib, cols, s0, exists)
        got = first_hit_by_solve(oracle_lib, cols, s0, exists)
        assert got == want
        assert want[0] is not None
        # the planted x and the first hit differ whenever the kernel lets an earlier solution exist
        multi += int(want[1] != x)
    assert multi > 0


def test_padding_slots_are_free_variables(oracle_lib):
    """A slot whose flip falls beyond N (zero column) is a valid alternative
    with no syndrome change: the earliest solution leaves it unset unless
    the canonical order reaches it first (v before the diagonal)."""
    N, K = 64, 32
    H = oracle_lib.parity_H(N, K)
    rng = np.random.default_rng(11)
    for trial in range(40):
        Sp = int(rng.integers(2, 7))
        cols, s0, exists = random_instance(rng, H, Sp, with_solution=True, pad_share=0.35)
        assert first_hit_by_solve(oracle_lib, cols, s0, exists) == first_hit_by_walk(oracle_lib, cols, s0, exists)


def test_no_solution_means_abandon_after_every_valid_tep(oracle_lib):
    """s(y) outside the span of the slot columns: no valid TEP is a codeword,
    and the walk ends at the total count (the cap is not reached)."""
    N, K = 128, 64
    H = oracle_lib.parity_H(N, K)
    rng = np.random.default_rng(13)
    for trial in range(20):
        Sp = int(rng.integers(1, 7))
        cols, _, exists = random_instance(rng, H, Sp, with_solution=True)
        # a syndrome with a bit outside every slot column's support
        s0 = np.zeros(H.shape[0], np.uint8)
        free = np.nonzero(~cols.any(axis=1))[0]
        if free.size == 0:
            continue
        s0[free[0]] = 1
        hit, _, total = first_hit_by_walk(oracle_lib, cols, s0, exists)
        assert hit is None and total == int(np.prod([[1, 2, 2, 4][[0, 1, 2, 7].index(int(e))] for e in exists]))
        assert first_hit_by_solve(oracle_lib, cols, s0, exists) == (None, None, total)
