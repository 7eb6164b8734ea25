"""Distributed HPL on a P x Q process grid -- TEST INFRASTRUCTURE ONLY.

A plain CPU model of the paper's multi-process algorithm, run as gloo ranks
(torch.distributed) with numpy arithmetic, to check that the distributed
schedule reaches the single-process oracle's pivots and factors.  The CUDA
library runs on one GPU; nothing here is on its path, and this module never
loads it.  Only the test suite may import it.

What it models (paper sections):
  - Sec. II, Fig. 1: the N x N matrix is split into NB x NB blocks, and block
    (I, J) lives on process (I mod P, J mod Q) of a P x Q grid (2D block-cyclic).
  - Sec. I, Fig. 2 (FACT): the process column that owns panel k factors it.
    For every column, each process finds its candidate (largest magnitude,
    smallest global row on ties) among its rows, and the candidates travel
    over the process column together with their rows' panel values (the
    all-reduce that carries the pivot row); every process then picks the same
    pivot, swaps, scales and updates its own rows.
  - Sec. I (LBCAST): the factored panel and its pivots are broadcast along
    each process row.
  - Sec. I (RS): the panel's interchanges are applied to the other columns: the
    rows that the swaps move are gathered over each process column (an
    Allgatherv of the moved rows) and every process writes the rows it owns.
  - Sec. I (UPDATE): the process row that owns block row k forms
    U12 = L11^-1 A12 and broadcasts it down its process column; every process
    updates A22 -= L21 U12 on its own rows and columns.
  - Sec. III-C (split update): each process's trailing columns are split into
    two sections; the row swaps of the second section are started as
    asynchronous collectives before the first section is updated and waited
    for after it, so the communication of one section overlaps the update of
    the other.

Layout: rank = p Q + q (row-major grid).  A process keeps its blocks packed
in a local Fortran array (its global rows in increasing order by its local
row index, likewise columns).  Pivots are 1-based global rows (LAPACK).
"""
from __future__ import annotations

import numpy as np
import torch
import torch.distributed as dist
from scipy.linalg import solve_triangular


def owned(n: int, nb: int, parts: int, idx: int) -> np.ndarray:
    """Global indices (increasing) of the rows (or columns) owned by process
    row (or column) idx of `parts` in the block-cyclic layout."""
    g = np.arange(n)
    return g[(g // nb) % parts == idx]


class Grid:
    """The P x Q process grid and its row and column communicators."""

    def __init__(self, P: int, Q: int):
        self.P, self.Q = P, Q
        self.rank = dist.get_rank()
        assert dist.get_world_size() == P * Q
        self.p, self.q = divmod(self.rank, Q)
        # every rank must create every group, in the same order
        self.col_groups = [dist.new_group([p * Q + q for p in range(P)]) for q in range(Q)]
        self.row_groups = [dist.new_group([p * Q + q for q in range(Q)]) for p in range(P)]
        self.col = self.col_groups[self.q]   # my process column (P ranks)
        self.row = self.row_groups[self.p]   # my process row (Q ranks)

    def rank_of(self, p: int, q: int) -> int:
        return p * self.Q + q


def _allgather(t: torch.Tensor, group, size: int, async_op: bool = False):
    out = [torch.empty_like(t) for _ in range(size)]
    work = dist.all_gather(out, t, group=group, async_op=async_op)
    return out, work


class DistLU:
    """The distributed right-looking LU with partial pivoting of Sec. I/II."""

    def __init__(self, grid: Grid, n: int, nb: int, A_full: np.ndarray, split: bool = True):
        self.g, self.n, self.nb, self.split = grid, n, nb, split
        self.rows = owned(n, nb, grid.P, grid.p)   # my global rows
        self.cols = owned(n, nb, grid.Q, grid.q)   # my global columns
        self.A = np.asfortranarray(A_full[np.ix_(self.rows, self.cols)].copy())
        self.ipiv = np.zeros(n, dtype=np.int32)
        self.row_pos = {int(r): i for i, r in enumerate(self.rows)}

    # ---------------------------------------------------------------- FACT
    def _fact(self, j0: int, j1: int, pc: np.ndarray):
        """Factor global columns j0..j1-1 (local columns pc) on my process
        column; returns (pivots of the panel, L11 as a jb x jb array)."""
        g, P = self.g, self.g.P
        jb = j1 - j0
        Pn = self.A[:, pc]  # my rows of the panel (a copy; written back below)
        for j in range(j0, j1):
            c = j - j0
            # my candidate among my rows >= j: largest |a|, first (smallest) row on ties
            sel = np.nonzero(self.rows >= j)[0]
            if sel.size:
                mags = np.abs(Pn[sel, c])
                i = int(np.argmax(mags))  # argmax returns the first maximum
                cand_val, cand_row, cand_vals = float(mags[i]), int(self.rows[sel[i]]), Pn[sel[i], :]
            else:
                cand_val, cand_row, cand_vals = -1.0, n_big(self.n), np.zeros(jb)
            # row j's current values, from its owner (for the swap)
            mine_j = j in self.row_pos
            jvals = Pn[self.row_pos[j], :] if mine_j else np.zeros(jb)
            msg = torch.from_numpy(np.concatenate([[cand_val, float(cand_row), 1.0 if mine_j else 0.0],
                                                   cand_vals, jvals]))
            parts, _ = _allgather(msg, g.col, P)
            best_v, best_r, pivv, rowj = -2.0, n_big(self.n), None, None
            for m in parts:
                v, r = float(m[0]), int(m[1])
                if v > best_v or (v == best_v and r < best_r):
                    best_v, best_r, pivv = v, r, m[3:3 + jb].numpy().copy()
                if float(m[2]) == 1.0:
                    rowj = m[3 + jb:3 + 2 * jb].numpy().copy()
            p_row = best_r
            self.ipiv[j] = p_row + 1
            if p_row != j:
                if mine_j:
                    Pn[self.row_pos[j], :] = pivv
                if p_row in self.row_pos:
                    Pn[self.row_pos[p_row], :] = rowj
            piv = pivv[c]
            if piv != 0.0:
                below = np.nonzero(self.rows > j)[0]
                if below.size:
                    Pn[below, c] = Pn[below, c] / piv
                    if c + 1 < jb:
                        Pn[np.ix_(below, np.arange(c + 1, jb))] -= np.outer(Pn[below, c], pivv[c + 1:])
        self.A[:, pc] = Pn
        # L11 (rows j0..j1-1 of the panel) to every process of the column
        top = np.nonzero((self.rows >= j0) & (self.rows < j1))[0]
        blk = np.zeros((jb, jb))
        if top.size:
            blk[self.rows[top] - j0, :] = Pn[top, :]
        parts, _ = _allgather(torch.from_numpy(blk), g.col, P)
        L11 = sum(t.numpy() for t in parts)
        return self.ipiv[j0:j1].copy(), L11

    # -------------------------------------------------------------- LBCAST
    def _lbcast(self, k: int, j0: int, j1: int, pc, piv, L11):
        """The panel (my rows x jb), its pivots and L11 along my process row."""
        g = self.g
        jb = j1 - j0
        qk = k % g.Q
        src = g.rank_of(g.p, qk)
        payload = np.zeros(len(self.rows) * jb + jb + jb * jb)
        if g.q == qk:
            payload[: len(self.rows) * jb] = self.A[:, pc].ravel(order="F")
            payload[len(self.rows) * jb: len(self.rows) * jb + jb] = piv
            payload[len(self.rows) * jb + jb:] = L11.ravel(order="F")
        t = torch.from_numpy(payload)
        if g.Q > 1:
            dist.broadcast(t, src=src, group=g.row)
        payload = t.numpy()
        Lp = payload[: len(self.rows) * jb].reshape((len(self.rows), jb), order="F")
        piv = payload[len(self.rows) * jb: len(self.rows) * jb + jb].astype(np.int32)
        L11 = payload[len(self.rows) * jb + jb:].reshape((jb, jb), order="F")
        self.ipiv[j0:j1] = piv
        return Lp, L11

    # ------------------------------------------------------------------ RS
    @staticmethod
    def _moves(j0: int, piv: np.ndarray):
        """Composed interchanges: {destination row: source row} of the rows they move."""
        cur = {}
        for t, pv in enumerate(piv):
            a, b = j0 + t, int(pv) - 1
            if a == b:
                continue
            va, vb = cur.get(a, a), cur.get(b, b)
            cur[a], cur[b] = vb, va
        return {d: s for d, s in cur.items() if d != s}

    def _rs_start(self, moves, lc):
        """Start the exchange of the moved rows on my local columns lc: every
        process contributes the sources it owns (an Allgatherv over the process
        column, here an all-gather of fixed-size messages)."""
        g = self.g
        srcs = sorted(set(moves.values()))
        buf = np.zeros((len(srcs), len(lc)))
        have = np.zeros(len(srcs))
        for i, s in enumerate(srcs):
            if s in self.row_pos:
                buf[i] = self.A[self.row_pos[s], lc]
                have[i] = 1.0
        msg = torch.from_numpy(np.concatenate([have, buf.ravel()]))
        parts, work = _allgather(msg, g.col, g.P, async_op=True)
        return (srcs, lc, parts, work)

    def _rs_finish(self, moves, state):
        srcs, lc, parts, work = state
        if work is not None:
            work.wait()
        ns = len(srcs)
        vals = {}
        for m in parts:
            arr = m.numpy()
            have, buf = arr[:ns], arr[ns:].reshape((ns, len(lc)))
            for i, s in enumerate(srcs):
                if have[i] == 1.0:
                    vals[s] = buf[i]
        for d, s in moves.items():
            if d in self.row_pos:
                self.A[self.row_pos[d], lc] = vals[s]

    # -------------------------------------------------------------- UPDATE
    def _update(self, k: int, j0: int, j1: int, Lp, L11, lc):
        """U12 = L11^-1 A12 by the owner of block row k, down the process
        column, then A22 -= L21 U12 on my rows and the local columns lc."""
        g = self.g
        jb = j1 - j0
        pk = k % g.P
        if len(lc) == 0:
            return
        U = np.zeros((jb, len(lc)))
        top = np.nonzero((self.rows >= j0) & (self.rows < j1))[0]
        if g.p == pk:
            U = solve_triangular(L11, self.A[np.ix_(top, lc)], lower=True, unit_diagonal=True)
            self.A[np.ix_(top, lc)] = U
        t = torch.from_numpy(np.ascontiguousarray(U))
        if g.P > 1:
            dist.broadcast(t, src=g.rank_of(pk, g.q), group=g.col)
        U = t.numpy()
        below = np.nonzero(self.rows >= j1)[0]
        if below.size:
            self.A[np.ix_(below, lc)] -= Lp[below, :] @ U

    # ----------------------------------------------------------------- run
    def factor(self):
        g, n, nb = self.g, self.n, self.nb
        for k in range((n + nb - 1) // nb):
            j0, j1 = k * nb, min(n, (k + 1) * nb)
            qk = k % g.Q
            pc = np.nonzero((self.cols >= j0) & (self.cols < j1))[0]  # my panel columns (if q == qk)
            piv, L11 = (self._fact(j0, j1, pc) if g.q == qk else (np.zeros(j1 - j0, dtype=np.int32),
                                                                     np.zeros((j1 - j0, j1 - j0))))
            Lp, L11 = self._lbcast(k, j0, j1, pc, piv, L11)
            moves = self._moves(j0, self.ipiv[j0:j1])
            left = np.nonzero(self.cols < j0)[0]
            right = np.nonzero(self.cols >= j1)[0]

            def rs(lc):
                return self._rs_start(moves, lc) if moves else None

            def rs_done(state):
                if state is not None:
                    self._rs_finish(moves, state)
            # RS left of the panel (LAPACK convention), then the split update
            rs_done(rs(left))
            if self.split and right.size > 1:
                h = right.size // 2
                s1, s2 = right[:h], right[h:]
                rs_done(rs(s1))
                pending = rs(s2)   # in flight during the update of s1
                self._update(k, j0, j1, Lp, L11, s1)
                rs_done(pending)
                self._update(k, j0, j1, Lp, L11, s2)
            else:
                rs_done(rs(right))
                self._update(k, j0, j1, Lp, L11, right)
        return self

    def gather(self) -> np.ndarray:
        """The packed factors, assembled on every rank (for the tests)."""
        g = self.g
        full = np.zeros((self.n, self.n))
        full[np.ix_(self.rows, self.cols)] = self.A
        t = torch.from_numpy(full)
        dist.all_reduce(t)  # every entry comes from exactly one process
        return t.numpy()


def n_big(n: int) -> int:
    """A row index larger than any real row (loses every tie)."""
    return n + 1


def factor(P: int, Q: int, n: int, nb: int, A_full: np.ndarray, split: bool = True):
    """Factor on the already initialised process group: (LU, ipiv) on every rank."""
    lu = DistLU(Grid(P, Q), n, nb, A_full, split=split).factor()
    return lu.gather(), lu.ipiv.copy()
