"""The mixed-precision solve at its full bench size: N = 65536, NB = 1536.

This is the configuration the bench line's mixed-precision block times (43
panels, the widest diagonal kernel, six levels of inverse products, the FP32
trailing matrix streamed 42 times).  For BF16 and FP8-E4M3:
  - the HPL scaled residual of the GMRES-IR solution is below 16, both by the
    library's Dot2 kernel and by the oracle, which regenerates A and b from the
    seed on the host (O(N^2), streamed, no N x N copy);
  - the forward error against the FP64 LU solve (partial pivoting) of the same
    system is within the bound the two residuals imply:
        ||x - x64|| / ||x64|| <= kappa_inf(A) n eps (s + s64)(1 + ||b|| / (||A|| ||x||))
    (each solution's error is at most kappa n eps s (...) by the definition of
    the scaled residual s), with kappa_inf(A) = ||A||_inf ||A^-1||_inf and
    ||A^-1||_inf estimated by Hager's method (Higham's refinement, as in
    LAPACK's xLACON) from solves with the FP64 factors; the estimate is a
    lower bound that is rarely off by more than a factor 3, so the test
    allows 10 times it.
"""
from __future__ import annotations

import numpy as np
import pytest
import torch

import oracle as O

pytestmark = pytest.mark.gpu

N, NB, SEED = 65536, 1536, 42
EPS = 2.0 ** -53


@pytest.fixture(scope="module")
def H():
    import __graft_entry__ as g
    g.build()
    import paper_2304_10397_gb300 as H
    assert torch.cuda.is_available()
    H.load_library()
    return H


def inv_norm_inf_estimate(H, LU, ipiv, n):
    """Estimate of ||A^-1||_inf = ||A^-T||_1 from the FP64 LU factors of A.

    Hager's 1-norm estimator applied to B = A^-T (B v = getrs('T'),
    B^T v = getrs('N')), with Higham's alternating test vector as a second
    candidate.  Both are lower bounds of the true norm."""
    def B(v):
        w = v.clone()
        H.getrs("T", LU, ipiv, w)
        return w

    def Bt(v):
        w = v.clone()
        H.getrs("N", LU, ipiv, w)
        return w

    x = torch.full((n,), 1.0 / n, device="cuda", dtype=torch.float64)
    est = 0.0
    for _ in range(5):
        y = B(x)
        est = max(est, float(y.abs().sum()))
        xi = torch.where(y >= 0, 1.0, -1.0).to(torch.float64)
        z = Bt(xi)
        j = int(z.abs().argmax())
        if float(z.abs()[j]) <= float(torch.dot(z, x)):
            break
        x = torch.zeros(n, device="cuda", dtype=torch.float64)
        x[j] = 1.0
    i = torch.arange(n, device="cuda", dtype=torch.float64)
    alt = torch.where(i % 2 == 0, 1.0, -1.0).to(torch.float64) * (1.0 + i / (n - 1))
    est2 = 2.0 * float(B(alt).abs().sum()) / (3.0 * n)
    return max(est, est2)


@pytest.fixture(scope="module")
def fp64_reference(H):
    A64, b = H.generate(N, SEED, dd=True)
    A = H.colmajor(N, N)
    A.copy_(A64)
    ipiv, info = H.getrf(A, 512)
    x64 = b.clone()
    H.getrs("N", A, ipiv, x64)
    H.sync_check()
    res64 = H.residual(N, SEED, x64, dd=True)
    ainv = inv_norm_inf_estimate(H, A, ipiv, N)
    del A, ipiv
    torch.cuda.empty_cache()
    assert int(info.item()) == 0 and res64[0] < 16
    return {"A64": A64, "b": b, "x64": x64, "res64": res64, "ainv": ainv}


@pytest.mark.parametrize("prec", [O.BF16, O.E4M3], ids=["bf16", "e4m3"])
def test_gmres_ir_full_size(H, fp64_reference, prec):
    ref = fp64_reference
    A64, b, x64 = ref["A64"], ref["b"], ref["x64"]
    LU, info = H.mxp_getrf(A64, NB, prec)
    x, st = H.gmres_ir(A64, LU, b, restart=50, max_outer=50, inner_tol=1e-10, target=16.0)
    H.sync_check()
    del LU
    torch.cuda.empty_cache()
    res = H.residual(N, SEED, x, dd=True)
    res_o = O.residual_seeded(N, SEED, x.cpu().numpy(), dd=True)
    fwd = float((x - x64).abs().max() / x64.abs().max())
    anorm, xnorm, bnorm = res_o[2], res_o[3], res_o[4]
    kappa = anorm * ref["ainv"]
    bound = 10 * kappa * N * EPS * (res_o[0] + ref["res64"][0]) * (1 + bnorm / (anorm * xnorm))
    print("N=%d prec=%d: outer %d inner %d residual %.4g (oracle %.4g), FP64 residual %.4g, "
          "kappa_inf ~ %.3g, FP64-relative error %.3g (bound %.3g)"
          % (N, prec, st["outer"], st["inner"], res[0], res_o[0], ref["res64"][0], kappa, fwd, bound))
    assert int(info.item()) == 0
    assert res[0] < 16 and res_o[0] < 16
    assert abs(res[0] - res_o[0]) <= 1e-6 * res_o[0]
    assert fwd <= bound
