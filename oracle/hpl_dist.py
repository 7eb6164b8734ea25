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
  - Sec. I-II (RS): the panel's interchanges are applied to the other
    columns.  The rows that leave the top block go from the process row that
    holds it to the owners of their destinations (Scatterv over the process
    column), and the jb rows that form the top block afterwards, the U rows,
    are gathered to every process of the column (Allgatherv).
  - Sec. I-II (UPDATE): every process forms U12 = L11^-1 U from the gathered U
    rows itself (so the phase needs no communication), the process row of the
    top block stores it, and every process updates A22 -= L21 U12 on its own
    rows and columns.
  - Sec. II (solve): b is appended to A as column N of an N x (N + 1)
    augmented system, so the elimination turns it into b_hat = L^-1 P b; the
    back substitution x = U^-1 b_hat runs block row by block row, the partial
    products of a block row summed over its process row to the owner of the
    diagonal block.
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
                 split: float = 0.5, b: np.ndarray | None = None):
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
        # with b, the N x (N + 1) augmented system of Sec. II: b is global column
        # N, distributed like any other column and carried through RS and UPDATE
        self.ncols = n + (b is not None)
        if b is not None:
            A_full = np.column_stack([A_full, np.asarray(b, dtype=np.float64)])
        self.rows = owned(n, nb, grid.P, grid.p)            # my global rows
        self.cols = owned(self.ncols, nb, grid.Q, grid.q)   # my global columns
        self.A = np.asfortranarray(A_full[np.ix_(self.rows, self.cols)].copy())
        self.Ucol = {}  # local column -> the panel's U rows (before DTRSM) on that column
        self.ipiv = np.zeros(n, dtype=np.int32)
        self.info = 0  # first zero pivot (1-based) seen by my FACT, LAPACK convention
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
            if piv == 0.0 and self.info == 0:
                self.info = j + 1
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

    def _rs_start(self, j0: int, j1: int, moves, lc):
        """Start RS of the panel at rows j0..j1-1 on my local columns lc (Sec. II):
        the rows that the interchanges move out of the top block go from the
        process row that holds the block to the processes that own their
        destinations (a Scatterv over the process column), and the jb rows that
        make up the top block afterwards, the U rows, are gathered to every
        process of the column (an Allgatherv), whether they move or not.
        Messages are padded to one size.  None when lc is empty (the same on
        every process of the column, which shares lc and the pivots)."""
        if len(lc) == 0:
            return None
        g, nb = self.g, self.nb
        pk = (j0 // nb) % g.P
        src_of_top = [moves.get(t, t) for t in range(j0, j1)]
        have = np.zeros(j1 - j0)
        buf = np.zeros((j1 - j0, len(lc)))
        for i, s in enumerate(src_of_top):
            if s in self.row_pos:
                buf[i] = self.A[self.row_pos[s], lc]
                have[i] = 1.0
        parts, w_ag = _allgather(torch.from_numpy(np.concatenate([have, buf.ravel()])), g.col, g.P,
                                 async_op=True)
        # the rows leaving the top block (their sources are top rows), by the
        # process row that owns each destination
        leaving = sorted(d for d in moves if not (j0 <= d < j1))
        per = [[d for d in leaving if (d // nb) % g.P == p] for p in range(g.P)]
        width = max(len(x) for x in per)
        out, w_sc = None, None
        if width:
            def pack(dests):
                t = np.zeros((width, len(lc)))
                for i, d in enumerate(dests):
                    t[i] = self.A[self.row_pos[moves[d]], lc]
                return torch.from_numpy(t.ravel())
            if g.P == 1:
                out = pack(per[0])
            else:
                out = torch.zeros(width * len(lc), dtype=torch.float64)
                lst = [pack(per[p]) for p in range(g.P)] if g.p == pk else None
                w_sc = dist.scatter(out, lst, src=g.rank_of(pk, g.q), group=g.col, async_op=True)
        return (j0, j1, lc, parts, w_ag, per[g.p], width, out, w_sc)

    def _rs_finish(self, state):
        """Wait for an RS, write the rows that land on my rows and keep the U
        rows of its columns for UPDATE."""
        if state is None:
            return
        j0, j1, lc, parts, w_ag, mine, width, out, w_sc = state
        w_ag.wait()
        if w_sc is not None:
            w_sc.wait()
        jb = j1 - j0
        U = np.zeros((jb, len(lc)))
        for m in parts:
            arr = m.numpy()
            have, buf = arr[:jb], arr[jb:].reshape((jb, len(lc)))
            U[have == 1.0] = buf[have == 1.0]
        for i, c in enumerate(lc):
            self.Ucol[int(c)] = U[:, i].copy()
        for t in range(j0, j1):
            if t in self.row_pos:
                self.A[self.row_pos[t], lc] = U[t - j0]
        if width:
            rows = out.numpy().reshape((width, len(lc)))
            for i, d in enumerate(mine):
                self.A[self.row_pos[d], lc] = rows[i]

    # -------------------------------------------------------------- UPDATE
    def _update(self, j0: int, j1: int, Lp, L11, lc):
        """UPDATE (Sec. II): every process of the column forms U12 = L11^-1 U
        from the U rows that RS gathered (the DTRSM, repeated on each, so the
        phase needs no communication), the process row that holds the top
        block stores it, and every process updates A22 -= L21 U12 on its rows
        below the panel and the local columns lc."""
        if len(lc) == 0:
            return
        U = np.stack([self.Ucol[int(c)] for c in lc], axis=1)
        U12 = solve_triangular(L11, U, lower=True, unit_diagonal=True)
        top = np.nonzero((self.rows >= j0) & (self.rows < j1))[0]
        if top.size:
            self.A[np.ix_(top, lc)] = U12[self.rows[top] - j0, :]
        below = np.nonzero(self.rows >= j1)[0]
        if below.size:
            self.A[np.ix_(below, lc)] -= Lp[below, :] @ U12

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
        n, nb, nc = self.n, self.nb, self.ncols
        nblk = (n + nb - 1) // nb
        if not self.lookahead:
            for k in range(nblk):
                j0, j1 = k * nb, min(n, (k + 1) * nb)
                Lp, L11 = self._lbcast_finish(self._panel(k))
                moves = self._moves(j0, self.ipiv[j0:j1])
                self.Ucol = {}
                outside = np.nonzero((self.cols < j0) | (self.cols >= j1))[0]
                self._rs_finish(self._rs_start(j0, j1, moves, outside))
                self._update(j0, j1, Lp, L11, self._cols_in(j1, nc))
                self.forms.append("plain")
            return self
        panel = self._lbcast_finish(self._panel(0))
        rs2, rs2_started = None, False  # the right section's RS for the current panel
        for k in range(nblk):
            j0, j1 = k * nb, min(n, (k + 1) * nb)
            j2 = min(n, j1 + nb)
            Lp, L11 = panel
            moves = self._moves(j0, self.ipiv[j0:j1])
            self.Ucol = {}
            done = self._cols_in(0, j0)  # factored columns: swapped too (LAPACK convention)
            la = self._cols_in(j1, j2)   # panel k + 1, the look-ahead
            if j2 <= self.c_split < n:
                sec1, sec2 = self._cols_in(j2, self.c_split), self._cols_in(self.c_split, nc)
                if not rs2_started:      # the first split iteration
                    rs2 = self._rs_start(j0, j1, moves, sec2)
                self._rs_finish(rs2)     # the right section's rows scattered
                self._rs_finish(self._rs_start(j0, j1, moves, la))
                self._update(j0, j1, Lp, L11, la)
                lb = self._panel(k + 1)  # FACT of panel k + 1; its LBCAST in flight
                rs1 = self._rs_start(j0, j1, moves, np.concatenate([done, sec1]))
                self._update(j0, j1, Lp, L11, sec2)  # UPDATE2, hiding LBCAST and RS1
                self._rs_finish(rs1)
                panel = self._lbcast_finish(lb)
                rs2 = self._rs_start(j1, j2, self._moves(j1, self.ipiv[j1:j2]), sec2)
                rs2_started = True
                self._update(j0, j1, Lp, L11, sec1)  # UPDATE1, hiding RS2 of panel k + 1
                self.forms.append("split")
            else:
                rest = self._cols_in(j2, nc)
                lc = np.concatenate([done, la, rest])
                if rs2_started:  # the last split iteration started the right section's RS
                    self._rs_finish(rs2)
                    lc = lc[self.cols[lc] < self.c_split]
                    rs2, rs2_started = None, False
                self._rs_finish(self._rs_start(j0, j1, moves, lc))
                self._update(j0, j1, Lp, L11, la)
                lb = self._panel(k + 1) if k + 1 < nblk else None
                self._update(j0, j1, Lp, L11, rest)  # hiding LBCAST
                if lb is not None:
                    panel = self._lbcast_finish(lb)
                self.forms.append("lookahead")
        return self

    # --------------------------------------------------------------- solve
    def solve(self) -> np.ndarray:
        """x = U^-1 b_hat on the augmented system (Sec. II), after factor():
        block rows from the last up, the processes of the block's process row
        sum their products U_kJ x_J (b_hat_k added by the process column that
        holds b) to the owner of the diagonal block (a reduce over the process
        row), which solves its triangle; x_k then goes to every process."""
        g, n, nb = self.g, self.n, self.nb
        if self.ncols != n + 1:
            raise ValueError("solve() needs the augmented system (b given)")
        x = np.zeros(n)
        qb = (n // nb) % g.Q
        bl = self._cols_in(n, n + 1)  # my local index of b, if I hold it
        for k in reversed(range((n + nb - 1) // nb)):
            j0, j1 = k * nb, min(n, (k + 1) * nb)
            pk, qk = k % g.P, k % g.Q
            t = torch.zeros(j1 - j0, dtype=torch.float64)
            if g.p == pk:
                top = np.nonzero((self.rows >= j0) & (self.rows < j1))[0]
                cj = self._cols_in(j1, n)
                acc = -(self.A[np.ix_(top, cj)] @ x[self.cols[cj]]) if cj.size else np.zeros(j1 - j0)
                if g.q == qb:
                    acc = self.A[top, bl[0]] + acc
                t = torch.from_numpy(np.ascontiguousarray(acc))
                if g.Q > 1:
                    dist.reduce(t, dst=g.rank_of(pk, qk), op=dist.ReduceOp.SUM, group=g.row)
                if g.q == qk:
                    dk = self._cols_in(j0, j1)
                    t = torch.from_numpy(solve_triangular(np.triu(self.A[np.ix_(top, dk)]), t.numpy()))
            if not (g.p == pk and g.q == qk):
                t = torch.zeros(j1 - j0, dtype=torch.float64)
            dist.broadcast(t, src=g.rank_of(pk, qk))
            x[j0:j1] = t.numpy()
        return x

    def global_info(self) -> int:
        """The first zero pivot over all panels (0 if none), on every rank."""
        t = torch.tensor([self.info if self.info else self.n + 1], dtype=torch.int64)
        dist.all_reduce(t, op=dist.ReduceOp.MIN)
        return 0 if int(t) == self.n + 1 else int(t)

    def gather(self) -> np.ndarray:
        """The packed N x N factors, assembled on every rank (for the tests)."""
        full = np.zeros((self.n, self.ncols))
        full[np.ix_(self.rows, self.cols)] = self.A
        t = torch.from_numpy(full)
        dist.all_reduce(t)  # every entry comes from exactly one process
        return t.numpy()[:, :self.n]


def n_big(n: int) -> int:
    """A row index larger than any real row (loses every tie)."""
    return n + 1


def factor(P: int, Q: int, n: int, nb: int, A_full: np.ndarray, lookahead: bool = True,
           split: float = 0.5, b: np.ndarray | None = None):
    """Factor on the already initialised process group: (LU, ipiv, the form
    of each iteration, x, info) on every rank, x = None without b, info the
    first zero pivot (1-based) or 0.  split is the right section's share of
    the blocks (0: no split)."""
    lu = DistLU(Grid(P, Q), n, nb, A_full, lookahead=lookahead, split=split, b=b).factor()
    x = lu.solve() if b is not None else None
    return lu.gather(), lu.ipiv.copy(), lu.forms, x, lu.global_info()
