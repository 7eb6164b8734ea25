"""The N > 1 host logic of bench.py ("replicas only": every rank solves its own
system; the job's value is the sum of the ranks' flops over the max of their
timed regions), exercised with the gloo backend on CPU, world size 2."""
from __future__ import annotations

import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, q):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    ws, r, lr = bench.dist_info()
    t_ms = [120.0, 150.0][rank]              # per-rank timed region
    flops = [1.0e12, 1.0e12][rank]           # per-rank work (same system size)
    tmax = bench.reduce_max(t_ms, world)
    ftot = bench.reduce_sum(flops, world)
    bench.barrier(world)
    q.put((rank, ws, r, tmax, ftot, ftot / (tmax * 1e-3) / 1e12))
    dist.destroy_process_group()


def test_replicas_reduction_gloo_world2():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=120) for _ in range(2))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, ws, r, tmax, ftot, value in out:
        assert ws == 2 and r == rank
        assert tmax == 150.0                   # max over ranks
        assert ftot == 2.0e12                  # whole-job work
        assert value == pytest.approx(2.0e12 / 0.150 / 1e12)


def test_single_rank_is_identity():
    import bench
    assert bench.reduce_max(3.5, 1) == 3.5 and bench.reduce_sum(2.0, 1) == 2.0
