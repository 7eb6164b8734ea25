"""The paper's multi-process HPL (2D block-cyclic P x Q grid, per-column pivot
exchange with the pivot row, LBCAST, row swaps by gathering the moved rows,
the split update of Sec. III-C) as gloo ranks on the CPU: it must reach the
single-process oracle's pivots exactly and its factors to rounding, on grids
1 x 2, 2 x 1 and 2 x 2, with ragged blocks (N not a multiple of NB P or NB Q)."""
from __future__ import annotations

import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp

import oracle as O


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, P, Q, n, nb, seed, split, q):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        from oracle import hpl_dist
        A, _ = O.generate(n, seed)
        LU, ipiv = hpl_dist.factor(P, Q, n, nb, A, split=split)
        if rank == 0:
            q.put((LU, ipiv))
    finally:
        dist.destroy_process_group()


def run_grid(P, Q, n, nb, seed, split=True):
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, P * Q, port, P, Q, n, nb, seed, split, q))
             for r in range(P * Q)]
    for p in procs:
        p.start()
    LU, ipiv = q.get(timeout=600)
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    return LU, ipiv


@pytest.mark.parametrize("P,Q,n,nb,split", [(1, 2, 100, 8, True), (2, 1, 100, 8, True), (2, 2, 150, 16, True),
                                            (2, 2, 77, 8, False)])
def test_distributed_lu_matches_the_oracle(P, Q, n, nb, split):
    seed = 42 + n
    LU, ipiv = run_grid(P, Q, n, nb, seed, split)
    A, b = O.generate(n, seed)
    LUo, ipo, info, st, mism = O.getrf(A)
    assert np.array_equal(ipiv, ipo)
    assert np.max(np.abs(LU - LUo)) <= 1e-12 * np.max(np.abs(LUo))
    assert O.factor_error(A, LU, ipiv) <= 10
    x = O.getrs("N", LU, ipiv, b)
    assert O.residual_dense(A, x, b)[0] < 16
