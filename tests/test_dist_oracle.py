"""The paper's multi-process HPL (2D block-cyclic P x Q grid, per-column pivot
exchange with the pivot row, LBCAST, row swaps by gathering the moved rows,
the look-ahead of Sec. III, Fig. 3 and the split update of Sec. III-C, Fig. 6)
as gloo ranks on the CPU: every rank must reach the single-process oracle's
pivots exactly and its factors to rounding, on grids from 1 x 2 to 4 x 2, with
ragged blocks (N not a multiple of NB P or NB Q), one panel narrower than NB,
NB = 1, and each iteration form (no look-ahead, look-ahead, split)."""
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


def _singular(n, seed):
    """The seeded system with column n // 3 set to zero: exactly singular, and
    the first zero pivot is at that column (LAPACK info = n // 3 + 1)."""
    A, b = O.generate(n, seed)
    A[:, n // 3] = 0.0
    return A, b


def _worker(rank, world, port, P, Q, n, nb, seed, lookahead, split, q, plant=False, singular=False):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        from oracle import hpl_dist
        A, b = _singular(n, seed) if singular else O.generate(n, seed)
        info = None
        if singular:
            LU, ipiv, forms, x, info = hpl_dist.factor(P, Q, n, nb, A, lookahead=lookahead, split=split)
        elif plant:
            class DropRightScatter(hpl_dist.DistLU):
                """A planted mistake: in the right section the rows that leave
                the top block are never written to their destinations."""

                def _rs_finish(self, state):
                    if state is not None and self.cols[state[2]].min() >= self.c_split:
                        j0, j1, lc, parts, w_ag, mine, width, out, w_sc = state
                        if w_sc is not None:
                            w_sc.wait()
                        state = (j0, j1, lc, parts, w_ag, mine, 0, out, None)
                    super()._rs_finish(state)
            lu = DropRightScatter(hpl_dist.Grid(P, Q), n, nb, A, lookahead=lookahead, split=split, b=b).factor()
            LU, ipiv, forms, x = lu.gather(), lu.ipiv.copy(), lu.forms, lu.solve()
        else:
            LU, ipiv, forms, x, info = hpl_dist.factor(P, Q, n, nb, A, lookahead=lookahead, split=split, b=b)
        q.put((rank, LU, ipiv, forms, x, info))
    finally:
        dist.destroy_process_group()


def run_grid(P, Q, n, nb, seed, lookahead=True, split=0.5, plant=False, singular=False):
    """Every rank's (LU, ipiv, forms, x, info), by rank."""
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, P * Q, port, P, Q, n, nb, seed, lookahead, split, q, plant,
                                                     singular))
             for r in range(P * Q)]
    for p in procs:
        p.start()
    out = {}
    for _ in procs:
        r, LU, ipiv, forms, x, info = q.get(timeout=600)
        out[r] = (LU, ipiv, forms, x, info)
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    return [out[r] for r in range(P * Q)]


# (P, Q, n, nb, look-ahead, split share, the forms the iterations must take)
CASES = [
    (1, 2, 100, 8, True, 0.5, {"split", "lookahead"}),
    (2, 1, 100, 8, True, 0.5, {"split", "lookahead"}),
    (2, 2, 150, 16, True, 0.5, {"split", "lookahead"}),
    (2, 2, 77, 8, False, 0, {"plain"}),
    (2, 2, 77, 8, True, 0, {"lookahead"}),
    (1, 3, 90, 8, True, 0.3, {"split", "lookahead"}),
    (3, 1, 90, 8, True, 0.7, {"split", "lookahead"}),
    (2, 3, 130, 8, True, 0.5, {"split", "lookahead"}),
    (2, 2, 7, 8, True, 0.5, {"lookahead"}),
    (2, 2, 24, 1, True, 0.5, {"split", "lookahead"}),
    (4, 2, 200, 8, True, 0.5, {"split", "lookahead"}),  # the paper's single-node grid (Sec. IV)
]


@pytest.mark.parametrize("P,Q,n,nb,lookahead,split,forms", CASES)
def test_distributed_lu_matches_the_oracle(P, Q, n, nb, lookahead, split, forms):
    seed = 42 + n
    res = run_grid(P, Q, n, nb, seed, lookahead, split)
    LU, ipiv, seen, x, info = res[0]
    assert set(seen) == forms and len(seen) == (n + nb - 1) // nb and info == 0
    for LUr, ipr, fr, xr, _ in res[1:]:  # every rank ends with the same factors, pivots and solution
        assert np.array_equal(ipr, ipiv) and np.array_equal(LUr, LU) and fr == seen
        assert np.array_equal(xr, x)
    A, b = O.generate(n, seed)
    LUo, ipo, info, st, mism = O.getrf(A)
    assert np.array_equal(ipiv, ipo)
    assert np.max(np.abs(LU - LUo)) <= 1e-12 * np.max(np.abs(LUo))
    assert O.factor_error(A, LU, ipiv) <= 10
    # the solution of the augmented system (b carried through the elimination,
    # then the distributed back substitution) against the oracle's solve
    xo = O.getrs("N", LUo, ipo, b)
    assert np.max(np.abs(x - xo)) <= 1e-10 * np.max(np.abs(xo))
    assert O.residual_dense(A, x, b)[0] < 16


def test_a_planted_schedule_mistake_is_caught():
    """Dropping the right section's Scatterv writes (the part of RS that the
    split update moves under UPDATE1) must break the agreement with the oracle."""
    n, nb, seed = 150, 16, 42 + 150
    LU, ipiv, forms, x, _ = run_grid(2, 2, n, nb, seed, True, 0.5, plant=True)[0]
    assert "split" in forms
    A, _ = O.generate(n, seed)
    LUo, ipo, info, st, mism = O.getrf(A)
    assert not np.array_equal(ipiv, ipo) or np.max(np.abs(LU - LUo)) > 1e-6 * np.max(np.abs(LUo))


def test_singular_matrix_reports_the_first_zero_pivot():
    """An exactly singular system: every rank reports the oracle's info (the
    first zero pivot, 1-based) and reaches its pivots and factors."""
    n, nb, seed = 90, 8, 17
    res = run_grid(2, 2, n, nb, seed, True, 0.5, singular=True)
    A, _ = _singular(n, seed)
    LUo, ipo, info_o, st, mism = O.getrf(A)
    assert info_o == n // 3 + 1
    for LU, ipiv, forms, x, info in res:
        assert info == info_o and np.array_equal(ipiv, ipo)
        assert np.max(np.abs(LU - LUo)) <= 1e-12 * np.max(np.abs(LUo))
