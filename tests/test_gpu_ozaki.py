"""GPU parity of the emulated FP64 trailing update (BF16 slice products on
tcgen05, after Ozaki et al. 2012) against the oracle of the same scheme.

  - hpl_dgemm_emulated is bitwise equal to the oracle: the splitting is exact
    on both sides, every level product is an exact integer (sums below 2^24 in
    FP32 accumulators), and the level sum and the final update are the same
    FP64 operations in the same order;
  - hpl_getrf_emulated (every trailing update emulated) meets the bars of the
    FP64 path: the oracle's pivots (up to the 1e-13 near-tie rule),
    ||PA - LU|| / (||A|| N eps) <= 10, scaled residual < 16; at the bench size
    N = 32768 the pivots equal those of the FP64 DGEMM path and the residual is
    checked by the oracle's streamed regeneration.
"""
from __future__ import annotations

import numpy as np
import pytest
import torch

import oracle as O
from tests import inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def H():
    import __graft_entry__ as g
    g.build()
    import paper_2304_10397_gb300 as H
    assert torch.cuda.is_available()
    H.load_library()
    return H


def dev(M, ld=None):
    import paper_2304_10397_gb300 as H
    T = H.colmajor(M.shape[0], M.shape[1], ld=ld)
    T.copy_(torch.from_numpy(np.ascontiguousarray(M)))
    return T


def host(T):
    torch.cuda.synchronize()
    return np.asfortranarray(T.cpu().numpy())


def levels_exact(k, s, beta):
    """k sum_{i+j=d} max|q_i| max|q_j| <= 2^24 for every kept level d."""
    for d in range(2, s + 2):
        bound = sum(2.0 ** (beta if i == 1 else beta - 1) * 2.0 ** (beta if d - i == 1 else beta - 1)
                    for i in range(1, d) if i <= s and d - i <= s)
        if k * bound > 2.0 ** 24:
            return False
    return True


def slice_params(k, slices):
    """The library's documented choice: (8, 7), (9, 6) or (11, 5) for slices = 0,
    else the widest beta <= 8 with exact levels and slices * beta <= 60."""
    if slices == 0:
        return next((s, b) for s, b in ((8, 7), (9, 6), (11, 5)) if levels_exact(k, s, b))
    return slices, next(b for b in range(8, 0, -1) if slices * b <= 60 and levels_exact(k, slices, b))


def oracle_update(A, B, Cm, slices):
    """The oracle with the library's passes over k (at most 1024 at a time)."""
    out = np.array(Cm, order="F", copy=True)
    k = A.shape[1]
    for k0 in range(0, k, 1024):
        k1 = min(k, k0 + 1024)
        s, beta = slice_params(k1 - k0, slices)
        out = O.ozaki_gemm(A[:, k0:k1], B[k0:k1, :], out, s, beta)
    return out


@pytest.mark.parametrize("m,n,k,extra", [(300, 500, 384, 0), (1000, 700, 64, 3), (129, 257, 100, 1),
                                         (77, 9, 1, 0), (4100, 300, 200, 0), (513, 640, 512, 2), (300, 260, 1100, 0)])
@pytest.mark.parametrize("slices", [0, 9])
@pytest.mark.parametrize("path", ["fused", "unfused"])
def test_dgemm_emulated_bitwise(H, m, n, k, extra, slices, path, monkeypatch):
    # fused: every level made and summed per 128 x 128 tile in one kernel;
    # unfused: the level products through HBM and a separate sum kernel
    if path == "unfused":
        monkeypatch.setenv("HPLGB_OZAKI_UNFUSED", "1")
    g = inputs.rng(m + n + k)
    A = inputs.uniform((m, k), seed=m + k) * 2.0 ** g.integers(-20, 5, (m, 1))
    B = inputs.uniform((k, n), seed=n + k) * 2.0 ** g.integers(-5, 20, (1, n))
    Cm = inputs.uniform((m, n), seed=m + n)
    A[min(2, m - 1), :] = 0.0  # a zero row (exponent 0)
    ref = oracle_update(A, B, Cm, slices)
    Ad, Bd, Cd = dev(A, m + extra), dev(B, k + extra), dev(Cm, m + extra)
    H.dgemm_emulated(Ad, Bd, Cd, slices=slices)
    H.sync_check()
    got = host(Cd)
    nbad = int(np.sum(got != ref))
    print("emulated (%s) m=%d n=%d k=%d slices=%d: %d of %d entries differ from the oracle; max |C - C_fp64|/|A||B| = %.3g"
          % (path, m, n, k, slices, nbad, m * n,
             np.max(np.abs(got - (Cm - A @ B)) / (np.abs(A) @ np.abs(B) + np.abs(Cm) + 1e-300))))
    assert nbad == 0


def test_dgemm_emulated_wide_range_rows_and_columns(H):
    # rows and columns whose magnitudes span 2^-300 .. 2^300 (each row/column
    # has its own exponent, so every one keeps its full precision)
    m, n, k = 256, 256, 128
    g = inputs.rng(5)
    A = inputs.uniform((m, k), seed=1) * 2.0 ** g.integers(-300, 300, (m, 1))
    B = inputs.uniform((k, n), seed=2) * 2.0 ** g.integers(-300, 300, (1, n))
    Cm = (A @ B) * 0.5
    ref = oracle_update(A, B, Cm, 0)
    Cd = dev(Cm)
    H.dgemm_emulated(dev(A), dev(B), Cd)
    assert np.array_equal(host(Cd), ref)


def compare_pivots(gp, A, rtol=1e-13):
    LU, oipiv, oinfo, st, mism = O.getrf(A, replay=gp, rtol=rtol)
    assert st == 0, "pivot mismatch beyond the near-tie rule"
    return LU, oinfo, mism


@pytest.mark.parametrize("n,nb,la", [(2048, 256, True), (1000, 96, False), (1500, 384, True)])
def test_getrf_emulated_vs_oracle(H, n, nb, la):
    seed = 42 + n
    A_d = H.colmajor(n, n)
    b_d = torch.empty(n, device="cuda", dtype=torch.float64)
    H.generate(n, seed, A=A_d, b=b_d)
    ipiv, info = H.getrf_emulated(A_d, nb, lookahead=la)
    x = b_d.clone()
    H.getrs("N", A_d, ipiv, x)
    H.sync_check()
    A, b = O.generate(n, seed)
    gp = ipiv.cpu().numpy()[:n]
    LU, oinfo, mism = compare_pivots(gp, A)
    LUg = host(A_d)
    ferr = O.factor_error(A, LUg, gp)
    res = O.residual_dense(A, x.cpu().numpy(), b)
    print("emulated getrf n=%d nb=%d: ferr %.3g residual %.3g near-tie replays %d max |LU - LU_orc| %.3g"
          % (n, nb, ferr, res[0], len(mism), np.max(np.abs(LUg - LU))))
    assert int(info.item()) == 0 == oinfo
    assert ferr <= 10 and res[0] < 16
    assert np.max(np.abs(LUg - LU)) <= 1e-10 * np.max(np.abs(LU))


@pytest.mark.parametrize("n,nb", [(4096, 384), (3000, 256)])
def test_getrf_emulated_lookahead_bitwise(H, n, nb, monkeypatch):
    # with the look-ahead the update of the remaining columns runs on fewer
    # SMs while FACT of the next panel runs beside it, and a second launch of
    # the update joins when FACT ends, taking tiles from the same counter:
    # that changes where each tile is computed, not how, so factors and
    # pivots are bitwise those without look-ahead, without the partition
    # (HPLGB_LA_SMS=0) and with another partition
    seed = 3 + n
    A_d = H.colmajor(n, n)
    outs = []
    for mode, la, sms in (("off", False, None), ("no partition", True, "0"), ("16 SMs", True, "16"),
                          ("default", True, None)):
        if sms is None:
            monkeypatch.delenv("HPLGB_LA_SMS", raising=False)
        else:
            monkeypatch.setenv("HPLGB_LA_SMS", sms)
        H.generate(n, seed, A=A_d, with_b=False)
        ipiv, info = H.getrf_emulated(A_d, nb, lookahead=la)
        H.sync_check()
        assert int(info.item()) == 0, mode
        outs.append((mode, A_d.clone(), ipiv.clone()))
    for mode, LU, ip in outs[1:]:
        nbad = int((LU != outs[0][1]).sum().item())
        print("emulated look-ahead (%s) n=%d nb=%d: %d entries differ from no look-ahead" % (mode, n, nb, nbad))
        assert torch.equal(ip, outs[0][2]) and nbad == 0, mode


def test_getrf_emulated_full_size_n32768(H):
    n, nb, seed = 32768, 384, 42
    A_d = H.colmajor(n, n)
    b_d = torch.empty(n, device="cuda", dtype=torch.float64)
    H.generate(n, seed, A=A_d, b=b_d)
    ipiv64, _ = H.getrf(A_d, nb)
    gp64 = ipiv64.cpu().numpy()[:n].copy()
    H.generate(n, seed, A=A_d, b=b_d)
    ipiv, info = H.getrf_emulated(A_d, nb)
    x = b_d.clone()
    H.getrs("N", A_d, ipiv, x)
    H.sync_check()
    gp = ipiv.cpu().numpy()[:n]
    assert int(info.item()) == 0
    assert np.array_equal(gp, gp64)  # no near-tie at this size: the same pivots as the FP64 path
    res_orc = O.residual_seeded(n, seed, x.cpu().numpy())
    res_gpu = H.residual(n, seed, x)
    assert res_orc[0] < 16 and np.allclose(res_gpu, res_orc, rtol=1e-6, atol=0)
    LUh = host(A_d)
    del A_d
    probe = O.factor_probe(n, seed, LUh, gp, inputs.rng(1).standard_normal(n))
    print("emulated n=32768: residual %.4g, probe of ||PA - LU|| %.4g" % (res_orc[0], probe))
    assert probe <= 10
