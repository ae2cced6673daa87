"""GPU tests of the serving loop: every result equals the same frame decoded
alone; admission by slots and by memory budget; concurrent submitters."""
from __future__ import annotations

import threading

import numpy as np
import pytest

import workloads as wl

pytestmark = pytest.mark.gpu

NS = (32, 64, 128, 256, 512, 1024)


@pytest.fixture(scope="module")
def env():
    import torch

    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2405_01808_gb300 as g

    g.build()
    codes = [g.Code.polar(n, n // 2) for n in NS]
    info = {}
    for n in NS:
        _, frozen = g.polar_H(n, n // 2)
        info[n] = np.setdiff1d(np.arange(n), frozen)
    return g, codes, info


def make_requests(g, mx, code_of_N):
    F = len(mx["N"])
    reqs = np.zeros(F, dtype=g.REQUEST_DTYPE)
    base = mx["symbols"].ctypes.data
    reqs["code"] = [code_of_N[int(n)] for n in mx["N"]]
    reqs["M"] = mx["M"]
    reqs["symbols"] = base + 8 * mx["sym_offset"].astype(np.uint64)
    reqs["tag"] = np.arange(F, dtype=np.uint64)
    return reqs


def alone(g, codes, code_of_N, mx, f, p):
    """The frame decoded by itself (one-frame call)."""
    import torch

    n, M = int(mx["N"][f]), int(mx["M"][f])
    L = wl.symbols_per_frame(n, M)
    o = mx["sym_offset"][f]
    sym = torch.from_numpy(np.ascontiguousarray(mx["symbols"][o:o + L]).reshape(1, L)).cuda()
    pp = g.Params.make(M=M, S=p.S, query_cap=p.query_cap)
    r = g.decode_symbols(codes[code_of_N[n]], pp, sym)
    torch.cuda.synchronize()
    return r["cw"].cpu().numpy().view(np.uint32)[0], int(r["queries"][0]), int(r["abandon"][0])


def run_all(srv, reqs, timeout_s=30.0):
    import time

    got = []
    i = 0
    t0 = time.time()
    while i < len(reqs):
        i += srv.submit(reqs[i:])
        got.append(srv.poll())
        assert time.time() - t0 < timeout_s
    srv.drain(timeout_s)
    while True:  # a poll returns a bounded number of results
        more = srv.poll()
        if not len(more):
            break
        got.append(more)
    return np.concatenate(got)


@pytest.mark.parametrize("membership", [0, 3, 5])  # TEP-by-TEP search; hash join; elimination
def test_results_equal_alone(env, membership):
    g, codes, info = env
    code_of_N = {n: i for i, n in enumerate(NS)}
    mx = wl.mixed_frames(60, 0, 3000, info, ebn0_range=(6.0, 14.0))
    p = g.Params.make(M=0, S=10, query_cap=1 << 20, membership=membership)
    srv = g.Server(codes, p, max_slots=4096, max_device_bytes=64 << 20, max_batch=512, n_streams=4)
    reqs = make_requests(g, mx, code_of_N)
    res = run_all(srv, reqs)
    st = srv.stats()
    srv.close()
    assert len(res) == 3000 and sorted(res["tag"].tolist()) == list(range(3000))
    assert st["completed"] == 3000 and st["errors"] == 0 and st["batches"] >= 2
    assert np.all(res["done_ns"] >= res["arrival_ns"])
    # every result equals the frame decoded alone (sampled: 300 frames, all kinds)
    by_tag = {int(r["tag"]): r for r in res}
    for f in np.linspace(0, 2999, 300).astype(int):
        cw, q, ab = alone(g, codes, code_of_N, mx, f, p)
        r = by_tag[int(f)]
        nw = int(mx["N"][f]) // 32
        assert (int(r["queries"]), int(r["abandon"])) == (q, ab), f
        assert np.array_equal(r["cw"][:nw], cw), f


@pytest.mark.parametrize("membership,step", [(0, 1), (3, 1), (0, 2)])
def test_long_frames_carried_equal_alone(env, membership, step):
    """resume_weight_step > 0: frames whose search outlasts the batch's weight
    window are continued from their device-resident cursors on a separate
    stream after the rest of their batch is reported; every result equals the
    frame decoded alone, and nothing is left in flight after the drain."""
    g, codes, info = env
    code_of_N = {n: i for i, n in enumerate(NS)}
    mx = wl.mixed_frames(62, step, 2000, info, ebn0_range=(4.0, 10.0))
    p = g.Params.make(M=0, S=10, query_cap=1 << 20, membership=membership)
    srv = g.Server(codes, p, max_slots=4096, max_device_bytes=64 << 20, max_batch=256, n_streams=4,
                   resume_weight_step=step)
    reqs = make_requests(g, mx, code_of_N)
    res = run_all(srv, reqs, timeout_s=60.0)
    st = srv.stats()
    srv.close()
    assert len(res) == 2000 and sorted(res["tag"].tolist()) == list(range(2000))
    assert st["completed"] == 2000 and st["errors"] == 0
    assert st["long_frames"] > 0 and st["resume_launches"] > 0
    assert st["long_live"] == 0 and st["live_slots"] == 0 and st["live_bytes"] == 0
    assert not (res["abandon"] == g.ABANDON_SUSPENDED).any()
    by_tag = {int(r["tag"]): r for r in res}
    # frames answered by the search stage (the carried ones among them) and a spread of the rest
    long_tags = res["tag"][res["queries"] > 631][:150].astype(np.int64)
    pick = np.unique(np.concatenate([long_tags, np.linspace(0, 1999, 150).astype(np.int64)]))
    for f in pick.tolist():
        cw, q, ab = alone(g, codes, code_of_N, mx, f, p)
        r = by_tag[f]
        nw = int(mx["N"][f]) // 32
        assert (int(r["queries"]), int(r["abandon"])) == (q, ab), f
        assert np.array_equal(r["cw"][:nw], cw), f


def test_admission_by_slots(env):
    g, codes, info = env
    code_of_N = {n: i for i, n in enumerate(NS)}
    mx = wl.mixed_frames(61, 0, 64, info, ebn0_range=(12.0, 14.0))
    p = g.Params.make(M=0, S=8, query_cap=1 << 16)
    srv = g.Server(codes, p, max_slots=8, max_device_bytes=16 << 20, n_streams=2)
    reqs = make_requests(g, mx, code_of_N)
    first = srv.submit(reqs)
    assert 1 <= first <= 8
    res = run_all(srv, reqs[first:])
    res = np.concatenate([res, srv.poll()])
    st = srv.stats()
    srv.close()
    assert st["rejected"] > 0 and st["admitted"] == 64
    assert st["live_slots"] == 0 and st["live_bytes"] == 0


def test_admission_by_memory(env):
    g, codes, info = env
    code_of_N = {n: i for i, n in enumerate(NS)}
    # N=1024 with QPSK: 512 symbols (4 KB) + record + outputs per request
    mx = wl.mixed_frames(62, 0, 40, info, ebn0_range=(12.0, 14.0), n_choices=(1024,), m_choices=(4,))
    p = g.Params.make(M=0, S=8, query_cap=1 << 16)
    budget = 5 * (8 * 512 + 144 + 128 + 5)
    srv = g.Server(codes, p, max_slots=1000, max_device_bytes=budget, n_streams=1)
    reqs = make_requests(g, mx, code_of_N)
    first = srv.submit(reqs)
    assert first == 5
    res = run_all(srv, reqs[first:])
    srv.close()


def test_concurrent_submitters(env):
    g, codes, info = env
    code_of_N = {n: i for i, n in enumerate(NS)}
    mx = wl.mixed_frames(63, 0, 4000, info, ebn0_range=(8.0, 14.0))
    p = g.Params.make(M=0, S=10, query_cap=1 << 20)
    srv = g.Server(codes, p, max_slots=2048, max_device_bytes=32 << 20, max_batch=256, n_streams=4)
    reqs = make_requests(g, mx, code_of_N)
    parts = np.array_split(np.arange(4000), 4)
    errors = []

    def feed(idx):
        try:
            i = 0
            while i < len(idx):
                i += srv.submit(reqs[idx[i:]])
        except Exception as e:  # pragma: no cover - reported below
            errors.append(e)

    ths = [threading.Thread(target=feed, args=(part,)) for part in parts]
    for t in ths:
        t.start()
    got = []
    while any(t.is_alive() for t in ths):
        got.append(srv.poll())
    for t in ths:
        t.join()
    srv.drain(30.0)
    got.append(srv.poll())
    res = np.concatenate(got)
    srv.close()
    assert not errors
    assert sorted(res["tag"].tolist()) == list(range(4000))


def test_batch_deadline(env):
    """params.deadline_ns bounds each batch: with a budget that has already run
    out when the search starts, every frame the preparation hands on comes back
    unsearched (abandon 5, the hard word, the preparation's query count) and
    the others as decoded alone; the codes' status words report the cuts."""
    g, codes, info = env
    code_of_N = {n: i for i, n in enumerate(NS)}
    mx = wl.mixed_frames(64, 0, 1500, info, ebn0_range=(4.0, 8.0))
    p = g.Params.make(M=0, S=10, query_cap=1 << 20, deadline_ns=1)
    srv = g.Server(codes, p, max_slots=4096, max_device_bytes=64 << 20, max_batch=512, n_streams=2)
    reqs = make_requests(g, mx, code_of_N)
    res = run_all(srv, reqs)
    st = srv.stats()
    srv.close()
    assert len(res) == 1500 and st["errors"] == 0
    cut = res["abandon"] == 5
    assert cut.sum() > 50
    p0 = g.Params.make(M=0, S=10, query_cap=1 << 20)
    for r in res[:: 7]:
        f = int(r["tag"])
        cw, q, ab = alone(g, codes, code_of_N, mx, f, p0)
        nw = int(mx["N"][f]) // 32
        if int(r["abandon"]) == 5:
            assert q > int(r["queries"])  # decoded alone it needs more than the preparation's queries
            assert ab != 5
        else:
            assert (int(r["queries"]), int(r["abandon"])) == (q, ab), f
            assert np.array_equal(r["cw"][:nw], cw), f
    cut_codes = {code_of_N[int(mx["N"][int(t)])] for t in res["tag"][cut]}
    for i, c in enumerate(codes):
        assert g.stream_status(c) == (g.E_TIMEOUT if i in cut_codes else 0), i


def test_drain_covers_batches_being_issued(env):
    """After drain returns, every admitted request's result is ready: one poll
    returns all of them (a batch the launcher is still issuing is counted)."""
    g, codes, info = env
    code_of_N = {n: i for i, n in enumerate(NS)}
    mx = wl.mixed_frames(65, 0, 2000, info, ebn0_range=(10.0, 14.0))
    p = g.Params.make(M=0, S=8, query_cap=1 << 16)
    for trial in range(5):
        srv = g.Server(codes, p, max_slots=4096, max_device_bytes=64 << 20, max_batch=256, n_streams=2)
        reqs = make_requests(g, mx, code_of_N)
        assert srv.submit(reqs) == 2000
        srv.drain(30.0)
        res = srv.poll()
        srv.close()
        assert len(res) == 2000, trial
