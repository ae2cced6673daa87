"""The multi-GPU bookkeeping on CPU ranks (gloo, world size 2): per-rank frame
shards are disjoint, and the aggregation sums units and takes the slowest
rank's time. No GPU and no collective on the decode path."""
from __future__ import annotations

import os
import socket

import numpy as np
import pytest


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out_dir):
    import torch.distributed as dist

    os.environ.update({"MASTER_ADDR": "127.0.0.1", "MASTER_PORT": str(port), "RANK": str(rank),
                       "WORLD_SIZE": str(world), "LOCAL_RANK": str(rank)})
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import workloads as wl
    from paper_2405_01808_gb300 import dist as gdist

    r, w, lr = gdist.rank_info()
    assert (r, w, lr) == (rank, world, rank)
    info = np.arange(64, 128)
    d = wl.qam_frames(2, gdist.shard_stream(rank, 0), 50, 128, info, 16, 8.0)
    np.save(os.path.join(out_dir, f"sym{rank}.npy"), d["symbols"])
    units, tmax = gdist.aggregate([10.0 * (rank + 1), 3.0], 5.0 + rank, dist)
    np.save(os.path.join(out_dir, f"agg{rank}.npy"), np.array(units + [tmax]))
    dist.barrier()
    dist.destroy_process_group()


def test_two_rank_sharding_and_aggregation(tmp_path):
    import torch.multiprocessing as mp

    port = _free_port()
    mp.start_processes(_worker, args=(2, port, str(tmp_path)), nprocs=2, join=True, start_method="spawn")
    a, b = np.load(tmp_path / "sym0.npy"), np.load(tmp_path / "sym1.npy")
    assert a.shape == b.shape and not np.array_equal(a, b)  # disjoint shards
    for r in range(2):
        agg = np.load(tmp_path / f"agg{r}.npy")
        assert agg.tolist() == [30.0, 6.0, 6.0]  # sums, and the slowest rank's time


def test_aggregate_single_process_is_identity():
    from paper_2405_01808_gb300 import dist as gdist

    assert gdist.aggregate([1.0, 2.0], 3.5, None) == ([1.0, 2.0], 3.5)
