"""The replica logic of bench.py on two CPU ranks (gloo, 127.0.0.1): the path has no exchange
step, so the ranks draw disjoint units, share none of them, and meet once to time the slowest
rank; the whole-job rate counts every rank's units over that time."""
import os
import socket

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    seeds = bench.rank_direction_seeds(rank, 8)
    members = bench.shard(range(13), rank, world)
    gathered = [None] * world
    dist.all_gather_object(gathered, (seeds, members))
    ms = 10.0 + 5.0 * rank                     # the slowest rank is the last one
    slowest = bench.max_over_ranks(ms, world, device="cpu")
    out[rank] = (gathered, slowest, bench.aggregate_rate(world, 8, 4, slowest))
    dist.destroy_process_group()


def test_two_replicas_on_gloo():
    world = 2
    port = _free_port()
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_rank_main, args=(world, port, out), nprocs=world, join=True)
        res = dict(out)
    for rank in range(world):
        gathered, slowest, rate = res[rank]
        seeds = [s for g in gathered for s in g[0]]
        members = [x for g in gathered for x in g[1]]
        assert len(set(seeds)) == len(seeds) == world * 8      # disjoint directions
        assert sorted(members) == list(range(13))              # every member exactly once
        assert slowest == 15.0                                  # max over ranks, same on both
        assert rate == pytest.approx(world * 8 * 4 / 15e-3)
