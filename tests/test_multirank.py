"""The multi-rank bench path on CPU: two gloo ranks, barrier and max-over-ranks
timing, and the whole-job aggregation (weak scaling: units of all ranks over
the slowest rank's time)."""
import os
import socket

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

import __graft_entry__  # noqa: F401


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    r, w, local = bench.dist_setup(world)
    bench.barrier(w, torch)
    secs = 1.0 + rank  # rank 1 is the slower one
    t = bench.max_over_ranks(secs, w, torch, torch.device("cpu"))
    value = bench.aggregate(units_per_rank=1e9, secs_max=t, world=w)
    q.put((r, w, t, value))
    dist.destroy_process_group()


def test_two_gloo_ranks():
    world = 2
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    got = sorted(q.get(timeout=10) for _ in range(world))
    for rank, (r, w, t, value) in enumerate(got):
        assert (r, w) == (rank, world)
        assert t == 2.0               # max over ranks
        assert value == 2 * 1e9 / 2.0 / 1e9  # both ranks' units over the slowest time
