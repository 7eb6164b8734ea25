"""GPU parity tests of the mixed-precision variant against the oracle.

  - quantization (tile exponents and BF16 / E4M3 codes): bit-exact;
  - tcgen05 trailing update: within the FP32 accumulation bound
    |C_gpu - C_ref| <= (K + 2) u32 (|C| + 2^-(eL+eU) |qL||qU|^T), u32 = 2^-24,
    against the exact product of the decoded codes (FP64);
  - the whole mixed-precision LU: exact on factors representable in both
    formats (dyadic L0 U0), and close to the oracle's MxP LU on the diagonally
    dominant system (normwise, a fraction of the format's unit roundoff);
  - GMRES-IR: HPL scaled residual < 16, forward error against the FP64
    unpivoted oracle solve stated and bounded.
"""
from __future__ import annotations

import numpy as np
import pytest
import torch

import oracle as O
from tests import inputs
from tests.mxp_compare import MXP_PANEL_BAR, panel_ratios, worst

pytestmark = pytest.mark.gpu
U32 = 2.0 ** -24


@pytest.fixture(scope="module")
def H():
    import __graft_entry__ as g
    g.build()
    import paper_2304_10397_gb300 as H
    assert torch.cuda.is_available()
    return H


def f32_dev(H, M, ld=None):
    T = H.colmajor(M.shape[0], M.shape[1], ld=ld, dtype=torch.float32)
    T.copy_(torch.from_numpy(np.ascontiguousarray(M, dtype=np.float32)))
    return T


E4M3_TABLE = None


def decode(codes, prec):
    global E4M3_TABLE
    codes = np.asarray(codes)
    if prec == O.BF16:
        return (codes.astype(np.uint32) << 16).view(np.float32).astype(np.float64)
    if E4M3_TABLE is None:
        E4M3_TABLE = np.array([O.e4m3_to_f32(c) for c in range(256)], dtype=np.float64)
    return E4M3_TABLE[codes.astype(np.int64) & 0xFF]


def kp_for(jb, prec):
    per = 64 if prec == O.BF16 else 128
    return (jb + per - 1) // per * per


def tiled_values(rows, cols, seed, by_rows):
    """FP32 values whose magnitude differs per 128-row (or -column) tile."""
    g = inputs.rng(seed)
    X = g.standard_normal((rows, cols))
    ext = rows if by_rows else cols
    for t in range((ext + 127) // 128):
        scale = 2.0 ** g.integers(-20, 20)
        if by_rows:
            X[t * 128:(t + 1) * 128, :] *= scale
        else:
            X[:, t * 128:(t + 1) * 128] *= scale
    return X.astype(np.float32)


@pytest.mark.parametrize("prec", [O.BF16, O.E4M3], ids=["bf16", "e4m3"])
@pytest.mark.parametrize("m2,jb", [(300, 96), (128, 128), (1000, 256), (5, 33)])
def test_quantize_bitexact(H, prec, m2, jb):
    kp = kp_for(jb, prec)
    L21 = tiled_values(m2, jb, seed=m2 + jb, by_rows=True)
    U12 = tiled_values(jb, m2, seed=m2 * 3 + jb, by_rows=False)
    ld = max(m2, jb) + 3
    W = np.zeros((ld, jb + m2), dtype=np.float32)
    W[:m2, :jb] = L21
    W[:jb, jb:] = U12
    Wd = f32_dev(H, W)
    eL, eU, qL, qU = H.mxp_quantize(prec, Wd[:m2, :jb], Wd[:jb, jb:], kp)
    torch.cuda.synchronize()
    oeL = O.tile_exps(L21, True, prec)
    oeU = O.tile_exps(U12, False, prec)
    assert np.array_equal(eL.cpu().numpy()[:len(oeL)], oeL)
    assert np.array_equal(eU.cpu().numpy()[:len(oeU)], oeU)
    cL = O.quantize(L21, True, prec, oeL)           # (m2, jb)
    cU = O.quantize(U12, False, prec, oeU)          # (jb, m2)
    gL = qL.cpu().numpy().view(np.uint16 if prec == O.BF16 else np.uint8).astype(np.uint16)
    gU = qU.cpu().numpy().view(np.uint16 if prec == O.BF16 else np.uint8).astype(np.uint16)
    assert np.array_equal(gL[:, :jb], cL)
    assert np.array_equal(gU[:, :jb], cU.T)
    assert not gL[:, jb:].any() and not gU[:, jb:].any()


def random_codes(rows, kp, prec, seed):
    """Codes (and exponents) of random tiled FP32 data, from the oracle."""
    X = tiled_values(rows, kp, seed=seed, by_rows=True)
    ex = O.tile_exps(X, True, prec)
    codes = O.quantize(X, True, prec, ex)  # (rows, kp) uint16
    return codes, ex


def codes_dev(codes, prec):
    """Row-major (C-contiguous) device copy of a (rows, kp) code array."""
    c = np.ascontiguousarray(codes)
    if prec == O.BF16:
        return torch.from_numpy(c.astype(np.uint16).view(np.int16)).cuda()
    return torch.from_numpy(c.astype(np.uint8)).cuda()


@pytest.mark.parametrize("prec", [O.BF16, O.E4M3], ids=["bf16", "e4m3"])
@pytest.mark.parametrize("m,n,ksteps", [(128, 256, 1), (300, 500, 3), (1024, 2048, 4), (77, 9, 2), (4100, 700, 2)])
@pytest.mark.parametrize("ld_kind", ["odd", "aligned"])
def test_tcgen05_update_parity(H, prec, m, n, ksteps, ld_kind):
    # an odd ldc takes the register epilogue, a 16-byte aligned one the TMA
    # epilogue (C staged through shared memory)
    kp = ksteps * (64 if prec == O.BF16 else 128)
    cL, eL = random_codes(m, kp, prec, seed=m + ksteps)
    cU, eU = random_codes(n, kp, prec, seed=n + 7 * ksteps)
    C = inputs.rng(5).standard_normal((m, n)).astype(np.float32)
    Cd = f32_dev(H, C, ld=m + 1 if ld_kind == "odd" else (m + 3) // 4 * 4)
    H.mxp_gemm(prec, codes_dev(cL, prec), codes_dev(cU, prec), torch.from_numpy(eL).cuda(),
               torch.from_numpy(eU).cuda(), Cd)
    torch.cuda.synchronize()
    got = Cd.cpu().numpy().astype(np.float64)
    dL, dU = decode(cL, prec), decode(cU, prec)
    scale = np.ldexp(1.0, -(eL[np.arange(m) // 128][:, None] + eU[np.arange(n) // 128][None, :]))
    ref = C.astype(np.float64) - scale * (dL @ dU.T)
    bound = (kp + 2) * U32 * (np.abs(C) + scale * (np.abs(dL) @ np.abs(dU).T))
    assert np.all(np.abs(got - ref) <= bound), np.max(np.abs(got - ref) / (bound + 1e-300))


@pytest.mark.parametrize("prec", [O.BF16, O.E4M3], ids=["bf16", "e4m3"])
@pytest.mark.parametrize("m,n,ksteps", [(128, 256, 1), (300, 500, 3), (1024, 2048, 4), (77, 9, 2), (4100, 700, 2),
                                        (640, 768, 12)])
def test_tcgen05_pair_update_parity(H, prec, m, n, ksteps, monkeypatch):
    # the SM-pair kernel (256 x 256 tiles over the two SMs of a cluster,
    # tcgen05 cta_group::2): the same bound, on shapes with an odd number of
    # 128-row tiles (the pair's second CTA beyond the last row) and ragged
    # columns; and against the single-SM kernel on the same inputs
    kp = ksteps * (64 if prec == O.BF16 else 128)
    cL, eL = random_codes(m, kp, prec, seed=m + ksteps)
    cU, eU = random_codes(n, kp, prec, seed=n + 7 * ksteps)
    C = inputs.rng(5).standard_normal((m, n)).astype(np.float32)
    ld = (m + 3) // 4 * 4
    args = (codes_dev(cL, prec), codes_dev(cU, prec), torch.from_numpy(eL).cuda(), torch.from_numpy(eU).cuda())
    monkeypatch.setenv("HPLGB_MXP_PAIR", "0")
    C1 = f32_dev(H, C, ld=ld)
    H.mxp_gemm(prec, *args, C1)
    monkeypatch.setenv("HPLGB_MXP_PAIR", "1")
    C2 = f32_dev(H, C, ld=ld)
    H.mxp_gemm(prec, *args, C2)
    H.sync_check()
    got = C2.cpu().numpy().astype(np.float64)
    dL, dU = decode(cL, prec), decode(cU, prec)
    scale = np.ldexp(1.0, -(eL[np.arange(m) // 128][:, None] + eU[np.arange(n) // 128][None, :]))
    ref = C.astype(np.float64) - scale * (dL @ dU.T)
    bound = (kp + 2) * U32 * (np.abs(C) + scale * (np.abs(dL) @ np.abs(dU).T))
    nbad = int((C1 != C2).sum().item())
    print("pair kernel m=%d n=%d K=%d prec=%d: %d entries differ from the single-SM kernel" % (m, n, kp, prec, nbad))
    assert np.all(np.abs(got - ref) <= bound), np.max(np.abs(got - ref) / (bound + 1e-300))


def gamma32(k):
    return k * U32 / (1 - k * U32)


@pytest.mark.parametrize("m,n,extra_ld", [(768, 1000, 0), (300, 517, 3), (128, 256, 0), (1, 5, 0), (2048, 300, 0),
                                          (65, 64, 1)])
def test_strsm_x3_vs_oracle(H, m, n, extra_ld):
    """U12 = L11^-1 A12 in FP32 on the tensor cores against the FP64 oracle
    substitution on the same FP32 inputs.  X^ = L^-1 by substitution has
    |X^ - L^-1| <= gamma_m |L^-1||L||L^-1|; the product from three BF16 pieces
    per operand (six partial products, FP32 accumulation over 6m terms) adds
    gamma_{6m+3} |X^||B|.  Twice the sum is the bar."""
    Lsrc, *_ = O.getrf(inputs.uniform((m, m), seed=m + 1))  # a pivoted L: |l_ij| <= 1
    L32 = np.asfortranarray(Lsrc.astype(np.float32))
    B32 = inputs.uniform((m, n), seed=n + 2).astype(np.float32)
    ref = O.trsm_llnu(L32.astype(np.float64), B32.astype(np.float64))
    Bd = f32_dev(H, B32, ld=m + extra_ld)
    H.strsm_llnu(f32_dev(H, L32, ld=m + extra_ld), Bd)
    got = Bd.cpu().numpy().astype(np.float64)
    L = np.tril(L32.astype(np.float64), -1) + np.eye(m)
    Li = np.abs(np.linalg.inv(L))
    aB = np.abs(B32.astype(np.float64))
    bound = 2 * (gamma32(m) * (Li @ (np.abs(L) @ (Li @ aB))) + gamma32(6 * m + 3) * (Li @ aB)) + 1e-30
    err = np.abs(got - ref)
    print("strsm x3 m=%d n=%d: max err / bound %.3g, max rel err %.3g"
          % (m, n, np.max(err / bound), np.max(err) / np.max(np.abs(ref))))
    assert np.all(err <= bound)


@pytest.mark.parametrize("prec", [O.BF16, O.E4M3], ids=["bf16", "e4m3"])
@pytest.mark.parametrize("n,nb", [(300, 128), (512, 256), (96, 32)])
def test_mxp_getrf_exact_on_representable_factors(H, prec, n, nb):
    # every step is exact on these factors: the panels, the U12 solve (by the
    # explicit inverse of each diagonal nb-block, which is I - N with N^2 = 0
    # here), the quantization and the tensor-core update
    L0, U0, A0 = inputs.dyadic_factors(n, seed=n + prec, block=nb)
    A = torch.from_numpy(np.asfortranarray(A0)).cuda()
    Ad = H.colmajor(n, n)
    Ad.copy_(torch.from_numpy(A0))
    LU, info = H.mxp_getrf(Ad, nb, prec)
    H.sync_check()
    W = LU.cpu().numpy()
    assert int(info.item()) == 0
    assert np.array_equal(np.tril(W, -1) + np.eye(n), L0.astype(np.float32))
    assert np.array_equal(np.triu(W), U0.astype(np.float32))
    del A


def check_panels_against_replay(W, A, nb, prec, label):
    """Every panel of the GPU's factors W against the oracle's factorization
    that quantizes the GPU's own L21 and U12 in each update (replay): the
    same quantized products on both sides, so what is left is FP32 arithmetic
    and each block must agree to MXP_PANEL_BAR of its largest entry.  The first
    panel has no earlier update at all: there both sides factor the same FP32
    input."""
    Wr, oinfo = O.mxp_getrf(A, nb, prec, replay=W)
    ratios = panel_ratios(W, Wr, nb)
    r, p, name = worst(ratios)
    print("%s: worst panel block %s of panel %d at %.3g of its largest entry (bar %.3g); first panel %s"
          % (label, name, p, r, MXP_PANEL_BAR, {k: "%.2g" % v for k, v in ratios[0].items()}))
    assert oinfo == 0
    assert r <= MXP_PANEL_BAR, (r, p, name)


@pytest.mark.parametrize("prec", [O.BF16, O.E4M3], ids=["bf16", "e4m3"])
@pytest.mark.parametrize("n,nb", [(1024, 256), (1000, 384), (700, 64)])
def test_mxp_getrf_vs_oracle(H, prec, n, nb):
    A, b = O.generate(n, 7, dd=True)
    Ad, _ = H.generate(n, 7, dd=True, with_b=False)
    LU, info = H.mxp_getrf(Ad, nb, prec)
    H.sync_check()
    W = LU.cpu().numpy()
    assert int(info.item()) == 0
    check_panels_against_replay(W, A, nb, prec, "mxp prec=%d n=%d nb=%d" % (prec, n, nb))
    # against the oracle's own run (its own quantization decisions): a code
    # that sits at a rounding boundary can go either way, so this is
    # normwise, and both reach the accuracy of the format
    Wo, oinfo = O.mxp_getrf(A, nb, prec)
    W64, Wo64 = W.astype(np.float64), Wo.astype(np.float64)
    rel = np.linalg.norm(W64 - Wo64) / np.linalg.norm(Wo64)

    def ferr(F):
        L = np.tril(F, -1) + np.eye(n)
        return np.linalg.norm(L @ np.triu(F) - A) / np.linalg.norm(A)
    print("  ||LU_gpu - LU_orc||/||LU_orc|| = %.3g, factor errors gpu %.3g oracle %.3g" % (rel, ferr(W64), ferr(Wo64)))
    assert oinfo == 0
    assert rel <= 2.0 ** -20
    assert ferr(W64) <= 2 * ferr(Wo64) + 1e-6


def test_mxp_getrf_widest_panel_vs_oracle(H):
    # NB = 2048, the widest diagonal block the kernels take (the most shared
    # memory per CTA, 64 substitution steps, six levels of inverse products),
    # then a ragged 52-column last panel
    n, nb, prec = 2100, 2048, O.E4M3
    A, b = O.generate(n, 5, dd=True)
    Ad, _ = H.generate(n, 5, dd=True, with_b=False)
    LU, info = H.mxp_getrf(Ad, nb, prec)
    H.sync_check()
    W = LU.cpu().numpy()
    assert int(info.item()) == 0
    check_panels_against_replay(W, A, nb, prec, "mxp nb=%d n=%d" % (nb, n))


@pytest.mark.parametrize("prec", [O.BF16, O.E4M3], ids=["bf16", "e4m3"])
def test_mxp_getrf_odd_leading_dimension(H, prec):
    # an odd leading dimension of the FP32 factors turns off every vector and
    # TMA path that needs 16-byte alignment (staged entries, piece splits,
    # quantization loads, the TMA C epilogue); the arithmetic is the same, so
    # the factors are bitwise those of the aligned layout
    n, nb = 777, 256
    Ad, _ = H.generate(n, 13, dd=True, with_b=False)
    LU1, info1 = H.mxp_getrf(Ad, nb, prec)
    LU2 = H.colmajor(n, n, dtype=torch.float32, ld=n + 1)
    LU2, info2 = H.mxp_getrf(Ad, nb, prec, LU32=LU2)
    H.sync_check()
    assert int(info1.item()) == 0 == int(info2.item())
    assert torch.equal(LU1, LU2)


@pytest.mark.parametrize("prec", [O.BF16, O.E4M3], ids=["bf16", "e4m3"])
def test_mxp_getrf_epilogue_paths_agree(H, prec, monkeypatch):
    # the tensor-core products have two epilogues (C through shared memory by
    # TMA, or through registers); both apply the same power-of-two scalings
    # and take the tile maxima for the quantization as they write, so the
    # whole factorization is bitwise the same either way (n = 1000: ragged
    # tiles and a short last panel)
    n, nb = 1000, 384
    Ad, _ = H.generate(n, 11, dd=True, with_b=False)
    LU1, info1 = H.mxp_getrf(Ad, nb, prec)
    H.sync_check()
    monkeypatch.setenv("HPLGB_MXP_REG_EPILOGUE", "1")
    LU2, info2 = H.mxp_getrf(Ad, nb, prec)
    H.sync_check()
    monkeypatch.delenv("HPLGB_MXP_REG_EPILOGUE")
    assert int(info1.item()) == 0 == int(info2.item())
    assert torch.equal(LU1, LU2)


@pytest.mark.parametrize("prec", [O.BF16, O.E4M3], ids=["bf16", "e4m3"])
@pytest.mark.parametrize("n,nb,diag_ctas", [(5000, 1536, None), (4608, 1536, None), (4096, 512, None),
                                            (4096, 512, "145")])
def test_mxp_getrf_lookahead_bitwise(H, prec, n, nb, diag_ctas, monkeypatch):
    # with the look-ahead, block column k+1 is updated first, the diagonal
    # kernel of panel k+1 runs on a second stream beside the rest of the
    # update, and two launches of the update (one per stream) share its tiles
    # through a counter; every entry is still the same product with K in the
    # same order, so the factors are bitwise those without it.  n = 5000 has a
    # ragged rest update and a last panel too narrow for the look-ahead;
    # n = 4608 ends with an update that is block column k+1 alone; "145" runs
    # the diagonal kernel on more CTAs than the fewest it needs.
    Ad, _ = H.generate(n, 17, dd=True, with_b=False)
    monkeypatch.setenv("HPLGB_MXP_LOOKAHEAD", "0")
    LU0, info0 = H.mxp_getrf(Ad, nb, prec)
    H.sync_check()
    monkeypatch.setenv("HPLGB_MXP_LOOKAHEAD", "1")
    if diag_ctas:
        monkeypatch.setenv("HPLGB_MXP_LA_DIAG_CTAS", diag_ctas)
    LU1, info1 = H.mxp_getrf(Ad, nb, prec)
    H.sync_check()
    assert int(info0.item()) == 0 == int(info1.item())
    nbad = int((LU0 != LU1).sum().item())
    print("mxp look-ahead n=%d nb=%d prec=%d: %d entries differ" % (n, nb, prec, nbad))
    assert nbad == 0


@pytest.mark.parametrize("prec", [O.BF16, O.E4M3], ids=["bf16", "e4m3"])
def test_gmres_ir_small(H, prec):
    n, nb, seed = 2048, 256, 42
    A64, b = H.generate(n, seed, dd=True)
    LU, info = H.mxp_getrf(A64, nb, prec)
    x, st = H.gmres_ir(A64, LU, b, restart=50, max_outer=50, inner_tol=1e-10, target=16.0)
    res = H.residual(n, seed, x, dd=True)
    Ah, bh = O.generate(n, seed, dd=True)
    LU64, oinfo = O.getrf_nopiv(Ah)
    x64 = O.getrs("N", LU64, None, bh)
    xg = x.cpu().numpy()
    fwd = np.max(np.abs(xg - x64)) / np.max(np.abs(x64))
    res_o = O.residual_dense(Ah, xg, bh)
    print("gmres-ir prec=%d n=%d: outer %d inner %d residual %.3g (oracle %.3g) fwd err %.3g"
          % (prec, n, st["outer"], st["inner"], res[0], res_o[0], fwd))
    assert res[0] < 16 and res_o[0] < 16
    # forward error implied by the scaled residual s: ||r|| <= s eps (||A|| ||x|| + ||b||) n, so
    # ||x - x*|| / ||x*|| <= kappa_inf(A) s n eps (1 + ||b|| / (||A|| ||x||)), twice for margin
    kappa = np.linalg.cond(Ah, np.inf)
    anorm, xnorm, bnorm = res_o[2], res_o[3], res_o[4]
    bound = 2 * kappa * res_o[0] * n * 2.0 ** -53 * (1 + bnorm / (anorm * xnorm))
    assert fwd <= bound, (fwd, bound)


@pytest.mark.parametrize("n,extra_ld", [(1500, 0), (1500, 1), (128, 0), (77, 3)])
def test_mxp_getrs_vs_oracle(H, n, extra_ld):
    # 16-byte aligned columns (float4 path) and odd leading dimensions (scalar
    # path); a ragged last 128-row block, a single full block, a single partial one
    A, b = O.generate(n, 3, dd=True)
    W, info = O.mxp_getrf(A, 256, O.BF16)
    ref = O.mxp_getrs(W, b)
    x = torch.from_numpy(b.copy()).cuda()
    H.mxp_getrs(f32_dev(H, W, ld=n + extra_ld), x)
    got = x.cpu().numpy()
    # FP32 substitution on x / max|x|: relative error a few u32 times the
    # condition of the triangular factors (diagonally dominant: small)
    assert np.max(np.abs(got - ref)) <= 1e-4 * np.max(np.abs(ref))
