"""The multi-rank host logic of bench.py on CPU: two gloo ranks take disjoint frame ranges
(weak scaling, no data exchanged) and agree on the slowest rank's time."""
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


def _worker(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    first = bench.rank_first_frame(512, rank, world)
    t = bench.max_over_ranks(10.0 + rank * 5.0, world)
    dist.barrier()
    q.put((rank, first, t))
    dist.destroy_process_group()


def test_two_gloo_ranks_shard_frames_and_take_max_time():
    world = 2
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=120) for _ in range(world))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert [o[1] for o in out] == [0, 512]          # disjoint frame ranges
    assert all(o[2] == 15.0 for o in out)           # every rank sees the max
    assert bench_single_rank_defaults()


def bench_single_rank_defaults():
    import bench
    return bench.rank_first_frame(512, 0, 1) == 0 and bench.max_over_ranks(3.0, 1) == 3.0
