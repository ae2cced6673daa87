"""Pins for the CPU oracle: each test checks the oracle against something other
than itself -- closed forms, brute force, hand-worked values, invariants -- so
that a dropped term, a wrong sign or index, or a transposed operand in the
oracle fails at least one of them. CPU only."""
from __future__ import annotations

import itertools
import math
import os

import numpy as np
import pytest

import workloads as wl

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


# ----------------------------------------------------------------------------
# helpers written independently of the oracle
# ----------------------------------------------------------------------------

def kron_G(N):
    """F^{(x)n} by numpy's Kronecker product (Def. II.1)."""
    F = np.array([[1, 0], [1, 1]], dtype=np.int64)
    G = np.array([[1]], dtype=np.int64)
    while G.shape[0] < N:
        G = np.kron(G, F)
    return G


def gf2_rank(A):
    A = (np.array(A, dtype=np.uint8) & 1).copy()
    rows, cols = A.shape
    r = 0
    for c in range(cols):
        piv = np.nonzero(A[r:, c])[0]
        if piv.size == 0:
            continue
        p = r + piv[0]
        A[[r, p]] = A[[p, r]]
        mask = A[:, c].astype(bool)
        mask[r] = False
        A[mask] ^= A[r]
        r += 1
        if r == rows:
            break
    return r


def esp(ks):
    """Coefficients of prod (1 + k x): the elementary symmetric polynomials."""
    poly = [1]
    for k in ks:
        nxt = poly + [0]
        for i in range(len(poly)):
            nxt[i + 1] += k * poly[i]
        poly = nxt
    return poly


def canonical_index(code, Sp, base=3, bits=2):
    """Closed-form canonical index of a TEP given by per-rank codes (`bits` bits
    per rank, 0 = unchanged, 1..base = the alternative; for the paper's order
    1 = h, 2 = v, 3 = diag)."""
    digits = [(code >> (bits * r)) & ((1 << bits) - 1) for r in range(Sp)]
    P = [r for r in range(Sp) if digits[r]]
    w = len(P)
    off = sum(math.comb(Sp, v) * base ** v for v in range(w))
    colex = sum(math.comb(p, j + 1) for j, p in enumerate(P))
    alpha = sum((digits[p] - 1) * base ** j for j, p in enumerate(P))
    return off + colex * base ** w + alpha


def gray(l):
    return l ^ (l >> 1)


# ----------------------------------------------------------------------------
# code construction (Def. II.1)
# ----------------------------------------------------------------------------

@pytest.mark.parametrize("N", [2, 4, 8, 32, 128])
def test_generator_is_kronecker_power_and_involution(oracle_lib, N):
    G = oracle_lib.generator_G(N).astype(np.int64)
    assert np.array_equal(G, kron_G(N))
    assert np.array_equal((G @ G) % 2, np.eye(N, dtype=np.int64))


def _bec_erasure_by_bruteforce(N, eps):
    """Erasure probability of each synthetic channel of G_N on a BEC(eps) under
    successive cancellation, by enumerating all 2^N erasure patterns: u_i is
    lost iff some u with u_<i = 0 and u_i = 1 encodes to zeros on every
    observed position."""
    G = kron_G(N)
    pe = np.zeros(N)
    for mask in range(1 << N):
        observed = [j for j in range(N) if not (mask >> j) & 1]
        p = eps ** (N - len(observed)) * (1 - eps) ** len(observed)
        for i in range(N):
            # unknowns u_{i+1..N-1}; equations sum_k u_k G[k][j] = G[i][j]
            A = np.array([[G[k][j] for k in range(i + 1, N)] + [G[i][j]] for j in observed],
                         dtype=np.uint8).reshape(len(observed), N - i)
            consistent = gf2_rank(A[:, :-1]) == gf2_rank(A) if A.size else True
            if consistent:
                pe[i] += p
    return pe


def test_bhattacharyya_matches_bec_bruteforce(oracle_lib):
    """Arikan's recursion is exact on the BEC; the oracle's parameters must equal
    the brute-force erasure probabilities (pins the index orientation)."""
    for N in (4, 8):
        eps = math.exp(-0.5)
        z = oracle_lib.bhattacharyya(N, 0.5, 0.0)
        assert np.allclose(z, _bec_erasure_by_bruteforce(N, eps), atol=1e-12, rtol=0)
    # capacity is conserved on the BEC: the mean parameter equals the input one
    z = oracle_lib.bhattacharyya(1024, 0.5, 0.0)
    assert abs(z.mean() - math.exp(-0.5)) < 1e-12


def test_frozen_set_n32(oracle_lib):
    """Bhattacharyya at 0 dB, R = 1/2, the 16 largest parameters frozen."""
    assert oracle_lib.frozen_set(32, 16).tolist() == [0, 1, 2, 3, 4, 5, 6, 7, 8, 9, 10, 12, 16, 17, 18, 20]
    for N in (32, 64, 128, 256, 512, 1024):
        f = oracle_lib.frozen_set(N, N // 2)
        z = oracle_lib.bhattacharyya(N, 0.5, 0.0)
        info = np.setdiff1d(np.arange(N), f)
        assert f.size == N // 2 and np.all(np.diff(f) > 0)
        assert z[f].min() >= z[info].max()


@pytest.mark.parametrize("N", [32, 64, 128, 256, 512, 1024])
def test_parity_matrix_annihilates_code(oracle_lib, N):
    K = N // 2
    H = oracle_lib.parity_H(N, K).astype(np.int64)
    f = oracle_lib.frozen_set(N, K)
    info = np.setdiff1d(np.arange(N), f)
    G = kron_G(N)
    assert not ((G[info] @ H.T) % 2).any()  # G_I H^T = 0
    assert gf2_rank(H) == N - K
    g = wl.rng(99, N)
    c = wl.random_codewords(g, 10000, N, info).astype(np.int64)
    assert not ((c @ H.T) % 2).any()


# ----------------------------------------------------------------------------
# demodulation (Def. II.2, Eq. 2, Def. III.1, Def. III.2)
# ----------------------------------------------------------------------------

def _read_hand_vectors():
    rows = []
    with open(os.path.join(GOLDEN, "demod_hand_vectors.txt")) as fh:
        for line in fh:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            t = line.split()
            rows.append(t)
    return rows


def _pt(s):
    return None if s == "none" else tuple(int(v) for v in s.split(","))


def test_qam_d_is_eq2(oracle_lib):
    for M, m in ((4, 1), (16, 2), (64, 3), (256, 4), (1024, 5), (4096, 6)):
        assert oracle_lib.qam_d(M) == pytest.approx(math.sqrt(3 * m / (M - 1)), rel=1e-15)
        # average symbol energy of the scaled odd-integer grid is 2m E_b
        side = int(math.isqrt(M))
        A = 2 * np.arange(side) - (side - 1)
        es = 2 * np.mean(A.astype(float) ** 2) * oracle_lib.qam_d(M) ** 2
        assert es == pytest.approx(2 * m, rel=1e-12)


@pytest.mark.parametrize("literal", [False, True])
def test_demod_hand_vectors(oracle_lib, literal):
    for t in _read_hand_vectors():
        M = int(t[0])
        rI, rQ = float(t[1]), float(t[2])
        AI, AQ = int(t[3]), int(t[4])
        Lx = float(t[15]) if literal else float(t[7])
        key = int(t[14]) if literal else int(t[8])
        nmask, hard = int(t[9]), int(t[10])
        nmask |= 32 * int(t[17] if literal else t[16])  # nearer alternative is vertical
        h, v, dg = _pt(t[11]), _pt(t[12]), _pt(t[13])
        d = math.sqrt(3 * (math.log2(M) / 2) / (M - 1))
        sym = np.array([[complex(rI * d, rQ * d)]], dtype=np.complex64)
        N = 32
        out = oracle_lib.demod(np.repeat(sym, 1, axis=1), M, N, literal=literal)
        side = int(math.isqrt(M))
        lI, lQ = int(out["hard_idx"][0, 0]) >> 8, int(out["hard_idx"][0, 0]) & 0xFF
        assert (2 * lI - (side - 1), 2 * lQ - (side - 1)) == (AI, AQ)
        assert out["hard_idx"][0, 0] == hard
        assert out["key"][0, 0] == key
        assert out["nmask"][0, 0] == nmask
        assert out["rel"][0, 0] == pytest.approx(Lx, abs=2e-6)
        # neighbours from the mask
        nm = out["nmask"][0, 0]
        dI = 1 if nm & 8 else -1
        dQ = 1 if nm & 16 else -1
        got_h = (AI + 2 * dI, AQ) if nm & 1 else None
        got_v = (AI, AQ + 2 * dQ) if nm & 2 else None
        got_d = (AI + 2 * dI, AQ + 2 * dQ) if nm & 4 else None
        assert (got_h, got_v, got_d) == (h, v, dg)


@pytest.mark.parametrize("M", [4, 16, 64, 256, 1024, 4096])
def test_demod_hard_point_is_nearest_point(oracle_lib, M):
    """Brute force: the hard point is the nearest of the M points on the
    quantised grid; exactly on a threshold the upper level is taken."""
    side = int(math.isqrt(M))
    g = np.random.default_rng(M)
    d = math.sqrt(3 * (math.log2(M) / 2) / (M - 1))
    r = g.uniform(-side - 2, side + 2, size=(4000, 2))
    # include exact thresholds and exact points
    r[:200, 0] = 2 * g.integers(-side // 2, side // 2 + 1, size=200)
    r[200:400, 1] = 2 * g.integers(-side // 2, side // 2 + 1, size=200) - 1
    sym = (r[:, 0] * d + 1j * r[:, 1] * d).astype(np.complex64).reshape(-1, 1)
    out = oracle_lib.demod(sym, M, 32)
    q = np.float32(256.0 / d)
    A = 2 * np.arange(side) - (side - 1)
    for axis, comp in ((0, sym.real), (1, sym.imag)):
        aq = np.clip(np.rint(comp.astype(np.float32) * q), -32768, 32767).astype(np.int64)[:, 0]
        dist = np.abs(256 * A[None, :] - aq[:, None])
        best = dist.min(axis=1, keepdims=True)
        cand = np.where(dist == best, np.arange(side)[None, :], -1)
        want = cand.max(axis=1)  # tie (threshold) -> upper level
        got = (out["hard_idx"][:, 0] >> 8) if axis == 0 else (out["hard_idx"][:, 0] & 0xFF)
        assert np.array_equal(got.astype(np.int64), want)


def test_demod_invariants(oracle_lib):
    M = 64
    side = 8
    g = np.random.default_rng(5)
    d = math.sqrt(3 * 3 / 63)
    r = g.uniform(-side - 3, side + 3, size=(5000, 2))
    sym = (r[:, 0] * d + 1j * r[:, 1] * d).astype(np.complex64).reshape(-1, 1)
    out = oracle_lib.demod(sym, M, 32)
    nm = out["nmask"][:, 0]
    k = ((nm & 1) > 0).astype(int) + ((nm & 2) > 0) + ((nm & 4) > 0)
    assert set(np.unique(k)) <= {0, 1, 3}
    # diag exists iff both h and v exist
    assert np.array_equal((nm & 4) > 0, ((nm & 1) > 0) & ((nm & 2) > 0))
    # inside the constellation square every axis has a neighbour
    inside = (np.abs(r[:, 0]) < side - 1) & (np.abs(r[:, 1]) < side - 1)
    assert np.all(k[inside] == 3)
    # the FP64 likelihood is sqrt(dI^2 + dQ^2) with d <= 1 inside
    assert np.all(out["rel"][inside, 0] <= math.sqrt(2) + 1e-9)


def test_demod_packs_gray_labels(oracle_lib):
    """Noise-free symbols demodulate to the transmitted coded bits."""
    for M in (4, 16, 64, 256, 1024, 4096):
        for N in (32, 128):
            info = oracle_lib.info_set(N, N // 2)
            g = wl.rng(7, M + N)
            c = wl.random_codewords(g, 50, N, info)
            tx = wl.qam_modulate(c, M).astype(np.complex64)
            out = oracle_lib.demod(tx, M, N)
            assert np.array_equal(out["y"], wl.pack_bits(c))


# ----------------------------------------------------------------------------
# TEP order (Alg. 2 Steps 2-4, Cor. III.1)
# ----------------------------------------------------------------------------

@pytest.mark.parametrize("Sp", [0, 1, 2, 3, 5, 8])
def test_tep_order_all_neighbours(oracle_lib, Sp):
    exists = np.full(Sp, 7, dtype=np.uint8)
    codes, total = oracle_lib.tep_order(exists)
    assert total == 4 ** Sp  # Cor. III.1 / Prop. III.1: 4^S patterns
    idx = [canonical_index(int(c), Sp) for c in codes]
    assert idx == list(range(4 ** Sp))
    w = np.array([sum(1 for r in range(Sp) if (int(c) >> 2 * r) & 3) for c in codes])
    for k in range(Sp + 1):
        assert np.sum(w == k) == math.comb(Sp, k) * 3 ** k
    # bit weight of the pattern: h and v flip one Gray bit, diag two
    bw = np.array([sum({0: 0, 1: 1, 2: 1, 3: 2}[(int(c) >> 2 * r) & 3] for r in range(Sp)) for c in codes])
    for b in range(2 * Sp + 1):
        assert np.sum(bw == b) == math.comb(2 * Sp, b)


def test_tep_order_partial_neighbours(oracle_lib):
    g = np.random.default_rng(11)
    for trial in range(30):
        Sp = int(g.integers(1, 9))
        exists = g.choice(np.array([0, 1, 2, 7], dtype=np.uint8), size=Sp)
        codes, total = oracle_lib.tep_order(exists)
        ks = [{0: 0, 1: 1, 2: 1, 7: 3}[int(e)] for e in exists]
        assert total == int(np.prod([1 + k for k in ks]))
        idx = [canonical_index(int(c), Sp) for c in codes]
        assert all(a < b for a, b in zip(idx, idx[1:]))  # canonical order
        # every valid pattern appears exactly once
        allowed = [[0] + [a for a in (1, 2, 3) if (int(exists[r]) >> (a - 1)) & 1] for r in range(Sp)]
        want = sorted(canonical_index(sum(d << 2 * r for r, d in enumerate(ds)), Sp)
                      for ds in itertools.product(*allowed))
        assert idx == want
        w = [sum(1 for r in range(Sp) if (int(c) >> 2 * r) & 3) for c in codes]
        assert [w.count(k) for k in range(Sp + 1)] == esp(ks)


@pytest.mark.parametrize("Sp", [0, 1, 2, 4, 7])
def test_tep_order_five_point_all_neighbours(oracle_lib, Sp):
    """Four alternatives per symbol (the five-point NNE model of Sec. II):
    5^S' patterns, C(S', w) 4^w of them with w altered symbols."""
    codes, total = oracle_lib.tep_order_n(np.full(Sp, 15, np.uint8), 4)
    assert total == 5 ** Sp
    idx = [canonical_index(int(c), Sp, base=4, bits=3) for c in codes]
    assert idx == list(range(5 ** Sp))
    w = np.array([sum(1 for r in range(Sp) if (int(c) >> 3 * r) & 7) for c in codes])
    for k in range(Sp + 1):
        assert np.sum(w == k) == math.comb(Sp, k) * 4 ** k


def test_tep_order_five_point_partial_neighbours(oracle_lib):
    """Edge and corner symbols (2 or 3 alternatives): the valid patterns are
    exactly the allowed products, in canonical order, counted by e_w(k)."""
    g = np.random.default_rng(12)
    for trial in range(30):
        Sp = int(g.integers(1, 7))
        exists = g.choice(np.array([15, 7, 11, 13, 14, 5, 10, 3, 12], dtype=np.uint8), size=Sp)
        codes, total = oracle_lib.tep_order_n(exists, 4)
        ks = [bin(int(e)).count("1") for e in exists]
        assert total == int(np.prod([1 + k for k in ks]))
        allowed = [[0] + [a for a in (1, 2, 3, 4) if (int(exists[r]) >> (a - 1)) & 1] for r in range(Sp)]
        want = sorted(canonical_index(sum(d << 3 * r for r, d in enumerate(ds)), Sp, base=4, bits=3)
                      for ds in itertools.product(*allowed))
        assert [canonical_index(int(c), Sp, base=4, bits=3) for c in codes] == want
        w = [sum(1 for r in range(Sp) if (int(c) >> 3 * r) & 7) for c in codes]
        assert [w.count(k) for k in range(Sp + 1)] == esp(ks)


def test_select_is_stable_sort(oracle_lib):
    g = np.random.default_rng(3)
    for _ in range(50):
        L = int(g.integers(1, 80))
        key = g.integers(0, 6, size=L).astype(np.uint32)  # many ties
        S = int(g.integers(0, 14))
        got = oracle_lib.select(key, S)
        want = np.lexsort((np.arange(L), key))[: min(S, L)]
        assert np.array_equal(got, want)


# ----------------------------------------------------------------------------
# decoding (Alg. 2 and GRAND-AB)
# ----------------------------------------------------------------------------

def _codebook(oracle_lib, N):
    K = N // 2
    info = oracle_lib.info_set(N, K)
    u = np.zeros((1 << K, N), dtype=np.uint8)
    ids = np.arange(1 << K)
    for b, pos in enumerate(info):
        u[:, pos] = (ids >> b) & 1
    return wl.polar_encode(u)


def test_decode_noise_free(oracle_lib):
    for M, N in ((4, 32), (16, 128), (64, 256), (256, 128)):
        info = oracle_lib.info_set(N, N // 2)
        H = oracle_lib.parity_H(N, N // 2)
        g = wl.rng(1, M)
        c = wl.random_codewords(g, 20, N, info)
        tx = wl.qam_modulate(c, M).astype(np.complex64)
        r = oracle_lib.decode_qam(H, tx, M, S=8, cap=1 << 16)
        assert np.all(r["queries"] == 1) and np.all(r["abandon"] == 0)
        assert np.array_equal(r["cw"], wl.pack_bits(c))


def test_grand_ab_is_ml_within_radius(oracle_lib):
    """GRAND-AB at N=32 against brute-force ML over all 2^16 codewords: with a
    codeword within Hamming distance 3 the decision is the first such codeword
    in (weight, colex) order of the error pattern; otherwise abandon."""
    N = 32
    book = _codebook(oracle_lib, N)
    H = oracle_lib.parity_H(N, 16)
    info = oracle_lib.info_set(N, 16)
    d = wl.bpsk_frames(1, 0, 300, N, info, 1.0)
    r = oracle_lib.decode_ab(H, d["symbols"], 3, 5489)
    y = (d["symbols"] < 0).astype(np.uint8)
    for f in range(300):
        e = book ^ y[f]
        wt = e.sum(axis=1)
        dmin = wt.min()
        if dmin <= 3:
            cands = e[wt == dmin]
            pos = [np.nonzero(x)[0].tolist() for x in cands]
            ranks = [sum(math.comb(p, j + 1) for j, p in enumerate(P)) for P in pos]
            best = cands[int(np.argmin(ranks))]
            want_cw = wl.pack_bits((y[f] ^ best)[None, :])[0]
            q = sum(math.comb(N, v) for v in range(dmin)) + min(ranks) + 1
            assert r["abandon"][f] == 0
            assert np.array_equal(r["cw"][f], want_cw)
            assert r["queries"][f] == q
        else:
            assert r["abandon"][f] == 1 and r["queries"][f] == 5489
            assert np.array_equal(r["cw"][f], wl.pack_bits(y[f][None, :])[0])


def _expected_symbol_level(book_ints, sym_frame, M, N, S, cap, literal=False, order=1):
    """Brute force for one frame, independent of the oracle's search: order the
    symbols by the quantised key, enumerate every valid TEP by the closed-form
    canonical index, build each candidate word from the Gray labels and look
    it up in the codebook (membership by lookup, not by syndrome).
    order 1: h, v, diag; 2: the single-axis alternative of the nearer axis
    first (nmask bit 32 = vertical nearer); 3: the four axis neighbours
    (toward on I, toward on Q, away on I, away on Q), base-4 digits."""
    import oracle as orc
    dm = orc.demod(sym_frame[None, :], M, N, literal=literal)
    L = sym_frame.size
    m = int(math.log2(M)) // 2
    lI = (dm["hard_idx"][0] >> 8).astype(int)
    lQ = (dm["hard_idx"][0] & 0xFF).astype(int)
    nm = dm["nmask"][0].astype(int)
    by_key = np.lexsort((np.arange(L), dm["key"][0]))
    Sp = min(S, L)
    sel = by_key[:Sp]

    def labels_to_bits(lab_I, lab_Q):
        bits = np.zeros(2 * m * L, dtype=np.uint8)
        for i in range(L):
            lab = (gray(lab_I[i]) << m) | gray(lab_Q[i])
            for k in range(2 * m):
                bits[2 * m * i + k] = (lab >> (2 * m - 1 - k)) & 1
        return bits[:N]

    side = 1 << m
    alts = []
    for r in range(Sp):
        i = sel[r]
        dI = 1 if nm[i] & 8 else -1
        dQ = 1 if nm[i] & 16 else -1
        # each alternative as a level move (move_I, move_Q)
        moves = {1: (dI, 0), 2: (0, dQ), 3: (dI, dQ)}
        ok = {1: bool(nm[i] & 1), 2: bool(nm[i] & 2), 3: bool(nm[i] & 4)}
        if order == 2 and nm[i] & 32:
            moves[1], moves[2] = moves[2], moves[1]
            ok[1], ok[2] = ok[2], ok[1]
        if order == 3:
            moves = {1: (dI, 0), 2: (0, dQ), 3: (-dI, 0), 4: (0, -dQ)}
            ok = {1: bool(nm[i] & 1), 2: bool(nm[i] & 2), 3: 0 <= lI[i] - dI < side, 4: 0 <= lQ[i] - dQ < side}
        opts = [0] + [a for a in sorted(moves) if ok[a]]
        alts.append((i, moves, opts))
    base, bits = (4, 3) if order == 3 else (3, 2)
    combos = []
    for ds in itertools.product(*[a[2] for a in alts]):
        code = sum(d_ << bits * r for r, d_ in enumerate(ds))
        combos.append((canonical_index(code, Sp, base=base, bits=bits), ds))
    combos.sort()
    n_valid = len(combos)
    for pos, (t, ds) in enumerate(combos, start=1):
        if pos > cap:
            break
        II, QQ = lI.copy(), lQ.copy()
        for (i, moves, _), dd in zip(alts, ds):
            if dd:
                II[i] += moves[dd][0]
                QQ[i] += moves[dd][1]
        x = labels_to_bits(II, QQ)
        xi = int(wl.pack_bits(x[None, :])[0].astype(np.uint64)[0]) if N == 32 else None
        if xi in book_ints:
            return wl.pack_bits(x[None, :])[0], pos, 0
    y = labels_to_bits(lI, lQ)
    return wl.pack_bits(y[None, :])[0], min(cap, n_valid), 1


@pytest.mark.parametrize("M,snr,S", [(4, 2.0, 8), (16, 6.0, 5), (64, 10.0, 4), (256, 14.0, 3), (1024, 19.0, 3),
                                     (4096, 23.0, 2)])
def test_symbol_level_matches_codebook_bruteforce(oracle_lib, M, snr, S):
    N = 32
    book = _codebook(oracle_lib, N)
    book_ints = set(wl.pack_bits(book)[:, 0].astype(np.uint64).tolist())
    H = oracle_lib.parity_H(N, 16)
    info = oracle_lib.info_set(N, 16)
    d = wl.qam_frames(3, M, 40, N, info, M, snr)
    cap = 4 ** S
    r = oracle_lib.decode_qam(H, d["symbols"], M, S, cap)
    n_ab = 0
    for f in range(40):
        cw, q, ab = _expected_symbol_level(book_ints, d["symbols"][f], M, N, S, cap)
        assert (int(r["abandon"][f]), int(r["queries"][f])) == (ab, q), f
        assert np.array_equal(r["cw"][f], cw)
        n_ab += ab
    assert 0 < n_ab < 40  # both outcomes exercised


@pytest.mark.parametrize("order,M,snr,S", [(2, 4, 2.0, 8), (2, 16, 6.0, 5), (2, 64, 9.0, 4),
                                           (3, 4, 2.0, 6), (3, 16, 6.0, 4), (3, 64, 9.0, 3)])
def test_order_variants_match_codebook_bruteforce(oracle_lib, order, M, snr, S):
    """The two order variants (nearer axis first; five-point NNE) against the
    codebook brute force at N=32, the whole TEP space within the cap."""
    N = 32
    book = _codebook(oracle_lib, N)
    book_ints = set(wl.pack_bits(book)[:, 0].astype(np.uint64).tolist())
    H = oracle_lib.parity_H(N, 16)
    info = oracle_lib.info_set(N, 16)
    d = wl.qam_frames(3, 100 * order + M, 40, N, info, M, snr)
    cap = (5 if order == 3 else 4) ** S
    r = oracle_lib.decode_qam(H, d["symbols"], M, S, cap, order=order)
    n_ab = 0
    for f in range(40):
        cw, q, ab = _expected_symbol_level(book_ints, d["symbols"][f], M, N, S, cap, order=order)
        assert (int(r["abandon"][f]), int(r["queries"][f])) == (ab, q), f
        assert np.array_equal(r["cw"][f], cw)
        n_ab += ab
    assert 0 < n_ab < 40


def _frame_with_moved_symbol(oracle_lib, want, place):
    """A 16-QAM N=128 frame received exactly on its points except one symbol:
    the first symbol whose transmitted amplitudes (A_I, A_Q) satisfy `want`
    is received at place(A_I, A_Q) (odd-integer units). Returns the
    codeword, the symbols and that symbol's index."""
    N, M = 128, 16
    info = oracle_lib.info_set(N, 64)
    c = wl.random_codewords(wl.rng(9, 0), 1, N, info)
    d = oracle_lib.qam_d(M)
    tx = np.round(wl.qam_modulate(c, M)[0] / d)
    i = next(j for j in range(tx.size) if want(int(tx[j].real), int(tx[j].imag)))
    rx = tx.copy()
    rx[i] = place(int(tx[i].real), int(tx[i].imag))
    return c, (rx * d).astype(np.complex64)[None, :], i


def test_nearer_axis_first_single_error(oracle_lib):
    """One symbol is received 0.2 past its Q threshold toward the centre
    (d_Q = 0.2, so the hard point is wrong on Q only) and 0.6 from its point
    toward the centre on I (d_I = 0.4). The transmitted point is then the
    vertical alternative of the least reliable symbol: query 3 in the
    paper's order (after h), query 2 when the nearer axis goes first."""
    N, M = 128, 16
    H = oracle_lib.parity_H(N, 64)
    c, s, i = _frame_with_moved_symbol(
        oracle_lib, lambda aI, aQ: True,
        lambda aI, aQ: complex(aI - 0.6 * np.sign(aI), aQ - 1.2 * np.sign(aQ)))
    dm = oracle_lib.demod(s, M, N)
    assert oracle_lib.select(dm["key"][0], 8)[0] == i
    assert dm["nmask"][0, i] & 32 and dm["nmask"][0, i] & 7 == 7
    a = oracle_lib.decode_qam(H, s, M, 8, 1 << 16, order=1)
    b = oracle_lib.decode_qam(H, s, M, 8, 1 << 16, order=2)
    for r in (a, b):
        assert r["abandon"][0] == 0 and np.array_equal(r["cw"][0], wl.pack_bits(c)[0])
    assert (int(a["queries"][0]), int(b["queries"][0])) == (3, 2)


def test_five_point_away_error(oracle_lib):
    """A symbol sent at (+-1, +-3) is received at (+-0.5, +-0.7): its hard
    point is (+-1, +-1) and the transmitted point is the neighbour on the Q
    axis away from the received value. With four alternatives per symbol
    (toward I, toward Q, away I, away Q, all present) it is the fourth
    alternative of rank 0: query 5."""
    N, M = 128, 16
    H = oracle_lib.parity_H(N, 64)
    c, s, i = _frame_with_moved_symbol(
        oracle_lib, lambda aI, aQ: abs(aI) == 1 and abs(aQ) == 3,
        lambda aI, aQ: complex(aI - 0.5 * np.sign(aI), 0.7 * np.sign(aQ)))
    dm = oracle_lib.demod(s, M, N)
    assert oracle_lib.select(dm["key"][0], 8)[0] == i
    r = oracle_lib.decode_qam(H, s, M, 8, 1 << 16, order=3)
    assert r["abandon"][0] == 0 and int(r["queries"][0]) == 5
    assert np.array_equal(r["cw"][0], wl.pack_bits(c)[0])
    # the paper's order cannot reach it at rank 0: its first hit, if any, is later
    p = oracle_lib.decode_qam(H, s, M, 8, 1 << 16, order=1)
    assert p["abandon"][0] == 1 or int(p["queries"][0]) > 4


def test_cap_boundary(oracle_lib):
    """A hit at exactly query = cap decodes; with cap one less it abandons."""
    N, M = 128, 16
    H = oracle_lib.parity_H(N, 64)
    info = oracle_lib.info_set(N, 64)
    d = wl.qam_frames(4, 0, 60, N, info, M, 8.0)
    r = oracle_lib.decode_qam(H, d["symbols"], M, 8, 1 << 16)
    f = int(np.nonzero((r["abandon"] == 0) & (r["queries"] > 3))[0][0])
    q = int(r["queries"][f])
    s = d["symbols"][f:f + 1]
    a = oracle_lib.decode_qam(H, s, M, 8, q)
    assert (a["abandon"][0], a["queries"][0]) == (0, q)
    assert np.array_equal(a["cw"][0], r["cw"][f])
    b = oracle_lib.decode_qam(H, s, M, 8, q - 1)
    y = oracle_lib.demod(s, M, N)["y"][0]
    assert (b["abandon"][0], b["queries"][0]) == (1, q - 1)
    assert np.array_equal(b["cw"][0], y)


def test_injected_error_at_least_reliable_symbol(oracle_lib):
    """Move the least reliable symbol of a noise-free-like frame to a
    neighbouring point: the search finds it within 1 + k_0 queries."""
    N, M = 128, 16
    H = oracle_lib.parity_H(N, 64)
    info = oracle_lib.info_set(N, 64)
    g = wl.rng(5, 0)
    c = wl.random_codewords(g, 30, N, info)
    tx = wl.qam_modulate(c, M)
    d = oracle_lib.qam_d(M)
    tx = tx + d * 0.05 * (g.standard_normal(tx.shape) + 1j * g.standard_normal(tx.shape))
    # push symbol 5 of each frame just across its nearest threshold toward 0
    for f in range(30):
        z = tx[f, 5] / d
        re = z.real - np.sign(z.real) * (abs(z.real) - abs(z.real) // 2 * 2 + 0.1) if abs(z.real) > 1 else -0.1 * np.sign(z.real)
        tx[f, 5] = d * complex(re, z.imag)
    sym = tx.astype(np.complex64)
    r = oracle_lib.decode_qam(H, sym, M, 8, 1 << 16)
    dm = oracle_lib.demod(sym, M, N)
    for f in range(30):
        sel = oracle_lib.select(dm["key"][f], 8)
        assert sel[0] == 5
        nm = int(dm["nmask"][f, 5])
        k0 = (nm & 1 > 0) + (nm & 2 > 0) + (nm & 4 > 0)
        assert r["abandon"][f] == 0
        assert np.array_equal(r["cw"][f], wl.pack_bits(c[f][None, :])[0])
        assert 1 < r["queries"][f] <= 1 + k0


def test_nonfinite_frame_is_not_searched(oracle_lib):
    N, M = 128, 16
    H = oracle_lib.parity_H(N, 64)
    info = oracle_lib.info_set(N, 64)
    d = wl.qam_frames(6, 0, 3, N, info, M, 8.0)
    s = d["symbols"].copy()
    s[1, 7] = np.complex64(complex(np.nan, 0.0))
    s[2, 0] = np.complex64(complex(0.5, np.inf))
    r = oracle_lib.decode_qam(H, s, M, 8, 1 << 16)
    assert r["abandon"].tolist()[1:] == [2, 2] and r["queries"].tolist()[1:] == [0, 0]
    ra = oracle_lib.decode_ab(oracle_lib.parity_H(32, 16), np.array([[np.nan] + [1.0] * 31], np.float32), 3, 5489)
    assert (ra["abandon"][0], ra["queries"][0]) == (2, 0)


def test_nonfinite_coordinate_reads_as_zero(oracle_lib):
    """A non-finite received coordinate is read as 0 for the hard word (R11).
    In 16-QAM, 0 lies exactly on the threshold between levels 1 and 2 and goes
    up to level 2 (amplitude +1, Gray label 11), so the I label of symbol 7 in
    the returned word is 1, 1 whatever was sent; every other symbol keeps its
    own hard decision."""
    N, M = 128, 16
    H = oracle_lib.parity_H(N, 64)
    d = wl.qam_frames(6, 1, 1, N, oracle_lib.info_set(N, 64), M, 30.0)
    s = d["symbols"].copy()
    s[0, 7] = np.complex64(complex(np.nan, s[0, 7].imag))
    r = oracle_lib.decode_qam(H, s, M, 8, 1 << 16)
    assert (r["abandon"][0], r["queries"][0]) == (2, 0)
    bits = ((r["cw"][0][:, None] >> np.arange(32, dtype=np.uint32)) & 1).reshape(-1)
    assert (bits[28], bits[29]) == (1, 1)  # symbol 7: bits 4*7 .. 4*7+3, I label first, MSB first
    zeroed = s.copy()
    zeroed[0, 7] = np.complex64(complex(0.0, s[0, 7].imag))
    assert np.array_equal(r["cw"][0], oracle_lib.demod(zeroed, M, N)["y"][0])


def test_bit_level_hard_decision_of_zero(oracle_lib):
    """Bit-level hard decision y = [r < 0]: samples of exactly +0.0 and -0.0 are
    bit 0. The all-zero codeword sent as +1 everywhere and received with two
    zero samples is its own hard word: decoded at query 1."""
    H = oracle_lib.parity_H(32, 16)
    r = np.ones((1, 32), np.float32)
    r[0, 3] = 0.0
    r[0, 9] = -0.0
    ra = oracle_lib.decode_ab(H, r, 3, 5489)
    assert (ra["abandon"][0], ra["queries"][0]) == (0, 1) and not ra["cw"][0].any()


def test_selection_ties_break_by_index(oracle_lib):
    """All 32 symbols of a 16-QAM frame sit 0.25 units from their point toward
    the centre (equal keys, exact in Q8.8, all k = 3); symbol 3 is received at
    the neighbouring point on the I axis. Ties must go to the lower index, so
    symbol 3 is rank 3 and its horizontal alternative is TEP t = 10: query 11."""
    N, M = 128, 16
    H = oracle_lib.parity_H(N, 64)
    info = oracle_lib.info_set(N, 64)
    g = wl.rng(8, 0)
    c = wl.random_codewords(g, 1, N, info)
    d = oracle_lib.qam_d(M)
    tx = np.round(wl.qam_modulate(c, M)[0] / d)  # odd-integer units
    rx = tx - 0.25 * np.sign(tx.real) - 0.25j * np.sign(tx.imag)
    # symbol 3 across the threshold toward the centre, 0.25 from the wrong point
    A = tx[3].real
    wrong = A - 2 * np.sign(A) if abs(A) == 3 else -A
    rx[3] = complex(wrong + 0.25 * np.sign(A), rx[3].imag)
    sym = (rx * d).astype(np.complex64)[None, :]
    keys = oracle_lib.demod(sym, M, N)["key"][0]
    assert len(set(keys.tolist())) == 1
    r = oracle_lib.decode_qam(H, sym, M, 10, 1 << 20)
    assert (int(r["abandon"][0]), int(r["queries"][0])) == (0, 11)
    assert np.array_equal(r["cw"][0], wl.pack_bits(c)[0])
