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
  - Sec. III, Fig. 3 (look-ahead): in iteration k the columns of panel k + 1
    are swapped and updated first, then factored by their process column, and
    their LBCAST is in flight while the rest of the update of panel k runs.
  - Sec. III-C, Fig. 6 (split update): the trailing columns are cut at a block
    boundary into a left section (the look-ahead and the columns up to the
    cut) and a right section of fixed width.  The left section's row exchange
    for panel k travels during the right section's update (UPDATE2); once
    panel k + 1 is factored, the right section's exchange for its pivots
    travels during the left section's update of panel k (UPDATE1) and is
    scattered at the start of the next iteration.  When the look-ahead reaches
    the cut, the iterations fall back to the plain look-ahead form.
  Overlap is modelled by asynchronous collectives that are started before a
  local update and waited for after it; on the CPU it changes nothing but the
  order of the steps, which is what the tests check against the oracle.

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

    def __init__(self, grid: Grid, n: int, nb: int, A_full: np.ndarray, lookahead: bool = True,
                 split: float = 0.5):
        if split and not lookahead:
            raise ValueError("the split update is built on the look-ahead")
        self.g, self.n, self.nb = grid, n, nb
        self.lookahead = lookahead
        self.forms = []  # the form each iteration took ("plain", "lookahead", "split")
        # The right section: the global columns from c_split on, a block
        # boundary, so that each process's n2 stays fixed and its n1 is a
        # multiple of NB (split = the right section's share of the blocks;
        # 0 turns the split update off).
        nblk = (n + nb - 1) // nb
        self.c_split = n if not split else min(n, nb * (nblk - int(split * nblk + 0.5)))
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
    def _lbcast_start(self, k: int, j0: int, j1: int, pc, piv, L11):
        """Start the broadcast of panel k (my rows x jb), its pivots and L11
        along my process row, from the process of the column that factored it."""
        g = self.g
        jb = j1 - j0
        nr = len(self.rows)
        payload = np.zeros(nr * jb + jb + jb * jb)
        if g.q == k % g.Q:
            payload[: nr * jb] = self.A[:, pc].ravel(order="F")
            payload[nr * jb: nr * jb + jb] = piv
            payload[nr * jb + jb:] = L11.ravel(order="F")
        t = torch.from_numpy(payload)
        work = None
        if g.Q > 1:
            work = dist.broadcast(t, src=g.rank_of(g.p, k % g.Q), group=g.row, async_op=True)
        return (t, work, j0, j1)

    def _lbcast_finish(self, state):
        """Wait for a panel broadcast; returns (my rows of the panel, L11) and
        records the panel's pivots."""
        t, work, j0, j1 = state
        if work is not None:
            work.wait()
        jb = j1 - j0
        nr = len(self.rows)
        payload = t.numpy()
        Lp = payload[: nr * jb].reshape((nr, jb), order="F").copy()
        self.ipiv[j0:j1] = payload[nr * jb: nr * jb + jb].astype(np.int32)
        L11 = payload[nr * jb + jb:].reshape((jb, jb), order="F").copy()
        return Lp, L11

    def _panel(self, k: int):
        """FACT of panel k on its process column, then its LBCAST started on
        every process (the factored values, pivots and L11)."""
        j0, j1 = k * self.nb, min(self.n, (k + 1) * self.nb)
        pc = self._cols_in(j0, j1)
        if self.g.q == k % self.g.Q:
            piv, L11 = self._fact(j0, j1, pc)
        else:
            piv, L11 = np.zeros(j1 - j0, dtype=np.int32), np.zeros((j1 - j0, j1 - j0))
        return self._lbcast_start(k, j0, j1, pc, piv, L11)

    def _cols_in(self, lo: int, hi: int) -> np.ndarray:
        """My local column indices whose global column lies in [lo, hi)."""
        return np.nonzero((self.cols >= lo) & (self.cols < hi))[0]

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
        column, here an all-gather of fixed-size messages).  None when there is
        nothing to move (the same on every process of the column, which shares
        lc and the pivots)."""
        g = self.g
        if not moves or len(lc) == 0:
            return None
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
        """Wait for an exchange and write the rows that land on my rows."""
        if state is None:
            return
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
        """All iterations.  Without look-ahead (Sec. II): FACT, LBCAST, RS and
        UPDATE of panel k, one after the other.  With it (Sec. III, Fig. 3) the
        columns of panel k + 1 are swapped and updated first, FACT of panel
        k + 1 and its LBCAST follow, and the update of the remaining columns
        runs while the broadcast is in flight.  With the split update
        (Sec. III-C, Fig. 6) the trailing columns are cut at c_split into a
        left section (the look-ahead and sec1) and a right section (sec2): the
        left section's exchange for panel k travels during UPDATE2 (sec2), and
        the right section's exchange for panel k + 1 during UPDATE1 (sec1) of
        panel k, until the look-ahead reaches c_split; from there the
        iterations take the plain look-ahead form."""
        n, nb = self.n, self.nb
        nblk = (n + nb - 1) // nb
        if not self.lookahead:
            for k in range(nblk):
                j0, j1 = k * nb, min(n, (k + 1) * nb)
                Lp, L11 = self._lbcast_finish(self._panel(k))
                moves = self._moves(j0, self.ipiv[j0:j1])
                outside = np.nonzero((self.cols < j0) | (self.cols >= j1))[0]
                self._rs_finish(moves, self._rs_start(moves, outside))
                self._update(k, j0, j1, Lp, L11, self._cols_in(j1, n))
                self.forms.append("plain")
            return self
        panel = self._lbcast_finish(self._panel(0))
        rs2, rs2_started = None, False  # the right section's exchange for the current panel
        for k in range(nblk):
            j0, j1 = k * nb, min(n, (k + 1) * nb)
            j2 = min(n, j1 + nb)
            Lp, L11 = panel
            moves = self._moves(j0, self.ipiv[j0:j1])
            done = self._cols_in(0, j0)  # factored columns: swapped too (LAPACK convention)
            la = self._cols_in(j1, j2)   # panel k + 1, the look-ahead
            if j2 <= self.c_split < n:
                sec1, sec2 = self._cols_in(j2, self.c_split), self._cols_in(self.c_split, n)
                if not rs2_started:      # the first split iteration
                    rs2 = self._rs_start(moves, sec2)
                self._rs_finish(moves, rs2)  # the right section's rows scattered
                self._rs_finish(moves, self._rs_start(moves, la))
                self._update(k, j0, j1, Lp, L11, la)
                lb = self._panel(k + 1)      # FACT of panel k + 1; its LBCAST in flight
                rs1 = self._rs_start(moves, np.concatenate([done, sec1]))
                self._update(k, j0, j1, Lp, L11, sec2)  # UPDATE2, hiding LBCAST and RS1
                self._rs_finish(moves, rs1)
                panel = self._lbcast_finish(lb)
                rs2 = self._rs_start(self._moves(j1, self.ipiv[j1:j2]), sec2)
                rs2_started = True
                self._update(k, j0, j1, Lp, L11, sec1)  # UPDATE1, hiding RS2 of panel k + 1
                self.forms.append("split")
            else:
                rest = self._cols_in(j2, n)
                lc = np.concatenate([done, la, rest])
                if rs2_started:  # the last split iteration started the right section's exchange
                    self._rs_finish(moves, rs2)
                    lc = lc[self.cols[lc] < self.c_split]
                    rs2, rs2_started = None, False
                self._rs_finish(moves, self._rs_start(moves, lc))
                self._update(k, j0, j1, Lp, L11, la)
                lb = self._panel(k + 1) if k + 1 < nblk else None
                self._update(k, j0, j1, Lp, L11, rest)  # hiding LBCAST
                if lb is not None:
                    panel = self._lbcast_finish(lb)
                self.forms.append("lookahead")
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


def factor(P: int, Q: int, n: int, nb: int, A_full: np.ndarray, lookahead: bool = True,
           split: float = 0.5):
    """Factor on the already initialised process group: (LU, ipiv, the form
    of each iteration) on every rank.  split is the right section's share of
    the blocks (0: no split)."""
    lu = DistLU(Grid(P, Q), n, nb, A_full, lookahead=lookahead, split=split).factor()
    return lu.gather(), lu.ipiv.copy(), lu.forms
