"""GPU tests of the differentiable solve (hand-written adjoint reusing the
stored LU factors and pivots): central finite differences on a tiny system,
torch.linalg.solve autograd (CPU, float64), and the closed-form FP64 oracle
gradient at the benchmarked size N=8192 with 64 right-hand sides."""
from __future__ import annotations

import numpy as np
import pytest
import torch

import oracle as O
from tests import inputs

pytestmark = pytest.mark.gpu
EPS = 2.0 ** -53


@pytest.fixture(scope="module")
def H():
    import __graft_entry__ as g
    g.build()
    import paper_2304_10397_gb300 as H
    from paper_2304_10397_gb300 import autograd  # noqa: F401
    return H


def test_adjoint_central_fd_n64(H):
    from paper_2304_10397_gb300.autograd import solve
    n, k, h = 64, 3, 1e-6
    A = inputs.uniform((n, n), seed=61) + np.eye(n)
    B = inputs.uniform((n, k), seed=62)
    W = inputs.uniform((n, k), seed=63)
    At = torch.tensor(A, device="cuda", requires_grad=True)
    Bt = torch.tensor(B, device="cuda", requires_grad=True)
    X = solve(At, Bt, 16)
    (X * torch.tensor(W, device="cuda")).sum().backward()
    dA = At.grad.cpu().numpy()
    dB = Bt.grad.cpu().numpy()

    def loss(Am, Bm):  # evaluated with the oracle (independent of the GPU path)
        LU, ip, *_ = O.getrf(Am)
        return float(np.sum(W * O.getrs("N", LU, ip, Bm)))

    g = inputs.rng(64)
    worst = 0.0
    for _ in range(8):
        i, j = g.integers(0, n, size=2)
        Ap, Am = A.copy(), A.copy()
        Ap[i, j] += h
        Am[i, j] -= h
        fd = (loss(Ap, B) - loss(Am, B)) / (2 * h)
        worst = max(worst, abs(fd - dA[i, j]) / max(1.0, abs(fd)))
        r, c = g.integers(0, n), g.integers(0, k)
        Bp, Bm = B.copy(), B.copy()
        Bp[r, c] += h
        Bm[r, c] -= h
        fd = (loss(A, Bp) - loss(A, Bm)) / (2 * h)
        worst = max(worst, abs(fd - dB[r, c]) / max(1.0, abs(fd)))
    print("adjoint vs central FD (h=1e-6, n=64): max rel err %.3g" % worst)
    assert worst <= 1e-7


def test_adjoint_vs_torch_linalg_solve(H):
    from paper_2304_10397_gb300.autograd import solve
    n, k = 200, 5
    A = inputs.uniform((n, n), seed=71)
    B = inputs.uniform((n, k), seed=72)
    W = inputs.uniform((n, k), seed=73)
    At = torch.tensor(A, device="cuda", requires_grad=True)
    Bt = torch.tensor(B, device="cuda", requires_grad=True)
    (solve(At, Bt, 64) * torch.tensor(W, device="cuda")).sum().backward()
    Ac = torch.tensor(A, requires_grad=True)
    Bc = torch.tensor(B, requires_grad=True)
    (torch.linalg.solve(Ac, Bc) * torch.tensor(W)).sum().backward()
    cond = np.linalg.cond(A, 1)
    tol = 10 * cond * n * EPS
    assert np.max(np.abs(At.grad.cpu().numpy() - Ac.grad.numpy())) <= tol * np.max(np.abs(Ac.grad.numpy()))
    assert np.max(np.abs(Bt.grad.cpu().numpy() - Bc.grad.numpy())) <= tol * np.max(np.abs(Bc.grad.numpy()))


def test_adjoint_vector_rhs(H):
    from paper_2304_10397_gb300.autograd import solve
    n = 300
    A = inputs.uniform((n, n), seed=81)
    b = inputs.uniform((n,), seed=82)
    At = torch.tensor(A, device="cuda", requires_grad=True)
    bt = torch.tensor(b, device="cuda", requires_grad=True)
    x = solve(At, bt, 64)
    x.sum().backward()
    LU, ip, *_ = O.getrf(A)
    lam = O.getrs("T", LU, ip, np.ones(n))
    assert np.allclose(bt.grad.cpu().numpy(), lam, rtol=1e-9, atol=1e-12)
    assert np.allclose(At.grad.cpu().numpy(), -np.outer(lam, O.getrs("N", LU, ip, b)), rtol=1e-8, atol=1e-12)


def test_adjoint_n8192_64rhs_vs_oracle(H):
    """The differentiable-solve configuration: N=8192, A from the seeded
    generator (seed 42), 64 right-hand sides B and upstream gradient W
    uniform [-0.5, 0.5) (seeds 43, 44)."""
    from paper_2304_10397_gb300.autograd import HplSolve
    n, k = 8192, 64
    A_gen, _ = H.generate(n, 42, with_b=False)
    A_d = A_gen.detach()  # a leaf (column-major view) that can require grad
    B = inputs.uniform((n, k), seed=43)
    W = inputs.uniform((n, k), seed=44)
    Bt = torch.tensor(B, device="cuda")
    Wt = torch.tensor(W, device="cuda")
    A_d.requires_grad_(True)
    Bt.requires_grad_(True)
    X = HplSolve.apply(A_d, Bt, 256, True)
    (X * Wt).sum().backward()
    torch.cuda.synchronize()
    # oracle: closed-form adjoint from the same factors (computed on the host)
    A, _ = O.generate(n, 42)
    # refactor on the GPU to hand the oracle the exact factors the adjoint used
    LUd = H.colmajor(n, n)
    LUd.copy_(A_d.detach())
    ipiv, info = H.getrf(LUd, 256)
    LU_g = np.asfortranarray(LUd.cpu().numpy())
    gp = ipiv.cpu().numpy()[:n]
    Xo = O.getrs("N", LU_g, gp, B)
    dAo, dBo = O.solve_adjoint(LU_g, gp, Xo, W)
    dA = A_d.grad.cpu().numpy()
    dB = Bt.grad.cpu().numpy()
    Xg = X.detach().cpu().numpy()
    relX = np.max(np.abs(Xg - Xo)) / np.max(np.abs(Xo))
    relB = np.max(np.abs(dB - dBo)) / np.max(np.abs(dBo))
    relA = np.max(np.abs(dA - dAo)) / np.max(np.abs(dAo))
    print("n=8192 k=64: rel err X %.3g dB %.3g dA %.3g" % (relX, relB, relA))
    # kappa-scaled bound of the solves: |dx| <= c kappa n eps |x| with kappa ~ 1e5 here
    assert relX <= 1e-7 and relB <= 1e-7 and relA <= 1e-7
