"""Panel-by-panel comparison of two sets of mixed-precision LU factors.

A test helper, not part of the method: it takes two FP32 factorizations of
the same n x n system with panels of nb columns (packed L and U, unit
diagonal of L implied) and reports, for every panel, the largest difference
in each of its four blocks -- the strictly lower part of the diagonal block
(L11), its upper part (U11), the block column below it (L21) and the block row
right of it (U12) -- divided by the largest magnitude in that block of the
reference.  Each block gets its own scale because their magnitudes differ by
orders (U11 carries the dominant diagonal, L21 entries are small).
"""
from __future__ import annotations

import numpy as np

U32 = 2.0 ** -24

# Bar of the panel comparison between the GPU's factors and the oracle
# replaying the GPU's quantized panels.  What separates the two is FP32
# arithmetic only: each panel's L11/U11 (blocked LU against unblocked
# elimination), its L21 = A21 U11^-1 and U12 = L11^-1 A12 (products of three
# BF16 pieces per operand, FP32 accumulation over K = nb terms, against
# substitution), and the FP32 rounding of every earlier update of the panel's
# entries (accumulated in TMEM against the exact sum rounded once).  Rounding
# errors of K-term FP32 sums grow like sqrt(K) u32 with high probability
# (Higham and Mary, SIAM J. Sci. Comput. 41, 2019); with K <= 2048 and a
# handful of such steps per entry the differences stay below 2^-17 of each
# block's largest entry (7.6e-6), which a planted relative error of 1e-5 in
# one block exceeds.
MXP_PANEL_BAR = 2.0 ** -17


def panel_ratios(W, Wref, nb):
    W = np.asarray(W, dtype=np.float64)
    R = np.asarray(Wref, dtype=np.float64)
    n = R.shape[0]
    out = []
    for k0 in range(0, n, nb):
        e = min(n, k0 + nb)
        D, Dr = W[k0:e, k0:e], R[k0:e, k0:e]
        blocks = {
            "L11": (np.tril(D, -1), np.tril(Dr, -1)),
            "U11": (np.triu(D), np.triu(Dr)),
            "L21": (W[e:, k0:e], R[e:, k0:e]),
            "U12": (W[k0:e, e:], R[k0:e, e:]),
        }
        r = {}
        for name, (got, ref) in blocks.items():
            if ref.size == 0:
                continue
            scale = float(np.max(np.abs(ref)))
            diff = float(np.max(np.abs(got - ref)))
            r[name] = diff / scale if scale > 0 else (0.0 if diff == 0 else np.inf)
        out.append(r)
    return out


def worst(ratios):
    """(largest ratio, panel index, block name)."""
    best = (0.0, -1, "")
    for p, r in enumerate(ratios):
        for name, v in r.items():
            if v > best[0]:
                best = (v, p, name)
    return best
