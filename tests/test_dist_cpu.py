"""Two-rank (gloo, CPU) checks of the replica-parallel host logic."""
import os
import socket

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

from paper_2401_02852_gb300 import dist as qdist


def test_shard_partitions_instances():
    for count in (0, 1, 7, 200):
        for world in (1, 2, 3, 8):
            parts = [qdist.shard(count, r, world) for r in range(world)]
            flat = sorted(i for p in parts for i in p)
            assert flat == list(range(count))
            assert max(map(len, parts)) - min(map(len, parts)) <= 1
    with pytest.raises(ValueError):
        qdist.shard(4, 2, 2)


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        mine = qdist.shard(10, rank, world)
        units = float(sum(2 ** 20 * 10 for _ in mine))  # amp-layers of n = 20, p = 10 instances
        secs = 1.0 + rank  # rank 1 is the slower one
        thr = qdist.job_throughput(units, secs)
        mx = qdist.max_over_ranks(secs)
        tot = qdist.sum_over_ranks(units)
        out[rank] = (thr, mx, tot, len(mine))
    finally:
        dist.destroy_process_group()


def test_two_rank_aggregation_gloo():
    world, port = 2, _free_port()
    mgr = mp.Manager()
    out = mgr.dict()
    mp.spawn(_worker, args=(world, port, out), nprocs=world, join=True)
    total_units = 10 * 2 ** 20 * 10
    for rank in range(world):
        thr, mx, tot, n_mine = out[rank]
        assert mx == 2.0 and tot == total_units
        assert thr == pytest.approx(total_units / 2.0)
        assert n_mine == 5


def test_single_process_falls_back_to_local_values():
    assert not dist.is_initialized()
    assert qdist.max_over_ranks(3.5) == 3.5
    assert qdist.job_throughput(10.0, 2.0) == 5.0
