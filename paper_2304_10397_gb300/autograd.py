"""Differentiable solve X = A^-1 B with a hand-written adjoint.

Forward: hpl_getrf (LU with partial pivoting) of a copy of A, then hpl_getrs
('N').  The factors, the pivots and X are kept for the backward pass.
Backward for an upstream gradient W = dL/dX:
    dB = A^-T W          -- hpl_getrs('T') on the stored factors and pivots
    dA = -dB X^T         -- hpl_outer_update, one fused rank-k FP64 product
Nothing is refactored.  (Not in the paper: it is the adjoint of the HPL
solve, for a loss sum(W .* X).)
"""
from __future__ import annotations

import torch

from . import colmajor, getrf, getrs, outer_update


def _cm_copy(M: torch.Tensor) -> torch.Tensor:
    out = colmajor(M.shape[0], M.shape[1], device=M.device)
    out.copy_(M)
    return out


class HplSolve(torch.autograd.Function):
    """X = A^-1 B (A: n x n, B: n x k, float64 CUDA tensors of any layout)."""

    @staticmethod
    def forward(ctx, A: torch.Tensor, B: torch.Tensor, nb: int = 256, lookahead: bool = True):
        if A.dim() != 2 or A.shape[0] != A.shape[1]:
            raise ValueError("A must be square")
        vec = B.dim() == 1
        B2 = B.unsqueeze(1) if vec else B
        LU = _cm_copy(A)
        ipiv, info = getrf(LU, nb, lookahead=lookahead)
        X = _cm_copy(B2)
        getrs("N", LU, ipiv, X)
        ctx.save_for_backward(LU, ipiv, X)
        ctx.vec = vec
        return X[:, 0] if vec else X

    @staticmethod
    def backward(ctx, W: torch.Tensor):
        LU, ipiv, X = ctx.saved_tensors
        W2 = W.unsqueeze(1) if ctx.vec else W
        lam = _cm_copy(W2.to(torch.float64))
        getrs("T", LU, ipiv, lam)                       # dB = A^-T W
        n = LU.shape[0]
        dA = colmajor(n, n, device=LU.device)
        outer_update(-1.0, lam, X, dA)                  # dA = -dB X^T
        dB = lam[:, 0] if ctx.vec else lam
        return dA, dB, None, None


def solve(A: torch.Tensor, B: torch.Tensor, nb: int = 256, lookahead: bool = True) -> torch.Tensor:
    return HplSolve.apply(A, B, nb, lookahead)
