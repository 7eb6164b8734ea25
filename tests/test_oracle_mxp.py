"""Pins for the mixed-precision part of the oracle (no GPU): the BF16 and
OCP FP8-E4M3 roundings against torch's conversions (library routines) and
hand-checked code points of the OCP specification, the exact power-of-two
scale rule, exact factorization of matrices whose factors are representable,
and the accuracy of the low-precision factors on the diagonally dominant
system."""
from __future__ import annotations

from fractions import Fraction

import numpy as np
import pytest

import oracle as O
from tests import inputs


def test_bf16_matches_torch():
    torch = pytest.importorskip("torch")
    g = inputs.rng(1)
    x = np.concatenate([g.standard_normal(20000).astype(np.float32) * 10.0 ** g.integers(-30, 30, 20000),
                        np.array([0.0, -0.0, 1.0, 1.00390625, 1.01171875, 3.3895314e38, 1e-40], dtype=np.float32)])
    x = x.astype(np.float32)
    ref = torch.from_numpy(x).to(torch.bfloat16).view(torch.int16).numpy().astype(np.uint16)
    got = np.array([O.f32_to_bf16(float(v)) for v in x], dtype=np.uint16)
    assert np.array_equal(got, ref)
    back = np.array([O.bf16_to_f32(int(h)) for h in got], dtype=np.float32)
    assert np.array_equal(back, torch.from_numpy(ref.view(np.int16)).view(torch.bfloat16).float().numpy())


def test_e4m3_matches_torch_in_range():
    torch = pytest.importorskip("torch")
    g = inputs.rng(2)
    x = (g.random(20000) * 2 - 1) * 448.0 * (2.0 ** -g.integers(0, 14, 20000))
    x = np.concatenate([x, [448.0, -448.0, 2.0 ** -9, 2.0 ** -10, 3 * 2.0 ** -11, 0.0, 1.0625, 1.1875, 240.0, 232.0]])
    x = x.astype(np.float32)
    ref = torch.from_numpy(x).to(torch.float8_e4m3fn).view(torch.uint8).numpy()
    got = np.array([O.f32_to_e4m3(float(v)) for v in x], dtype=np.uint8)
    assert np.array_equal(got, ref)


def test_e4m3_spec_code_points():
    # OCP 8-bit floating point specification, E4M3: bias 7, max 448, min subnormal 2^-9
    assert O.f32_to_e4m3(1.0) == 0x38
    assert O.f32_to_e4m3(-1.0) == 0xB8
    assert O.f32_to_e4m3(448.0) == 0x7E
    assert O.f32_to_e4m3(500.0) == 0x7E  # saturating
    assert O.f32_to_e4m3(2.0 ** -9) == 0x01
    assert O.f32_to_e4m3(2.0 ** -6) == 0x08  # smallest normal
    assert O.f32_to_e4m3(1.0625) == 0x38  # tie -> even (1.000)
    assert O.f32_to_e4m3(1.1875) == 0x3A  # tie -> even (1.010)
    for c in range(256):
        if (c & 0x7F) == 0x7F:
            assert np.isnan(O.e4m3_to_f32(c))
        else:
            assert O.f32_to_e4m3(O.e4m3_to_f32(c)) == (c if c != 0x80 else 0x80)


def test_scale_exp_is_the_largest_power():
    g = inputs.rng(3)
    for amax in list(g.random(300) * 10.0 ** g.integers(-20, 20, 300)) + [448.0, 1.0, 0.875, 2.0 ** -30]:
        for qm in (1.0, 448.0):
            e = O.scale_exp(float(amax), qm)
            a = Fraction(float(amax))
            assert a * Fraction(2) ** e <= qm < a * Fraction(2) ** (e + 1)
    assert O.scale_exp(0.0, 448.0) == 0


def test_quantize_tiles_layout():
    g = inputs.rng(4)
    X = (g.standard_normal((300, 40)) * 3).astype(np.float32, order="F")
    X[130, 7] = 100.0  # second row tile gets a smaller exponent
    ex = O.tile_exps(X, True, O.E4M3)
    assert len(ex) == 3 and ex[1] == O.scale_exp(100.0, 448.0)
    q = O.quantize(X, True, O.E4M3, ex)
    assert q[130, 7] == O.f32_to_e4m3(100.0 * 2.0 ** ex[1])
    exc = O.tile_exps(X, False, O.BF16)
    assert len(exc) == 1


@pytest.mark.parametrize("prec", [O.BF16, O.E4M3])
@pytest.mark.parametrize("n,nb", [(64, 16), (300, 128), (260, 256)])
def test_mxp_exact_on_representable_factors(prec, n, nb):
    L0, U0, A0 = inputs.dyadic_factors(n, seed=n + prec)
    W, info = O.mxp_getrf(A0, nb, prec)
    assert info == 0
    assert np.array_equal(np.tril(W, -1) + np.eye(n), L0.astype(np.float32))
    assert np.array_equal(np.triu(W), U0.astype(np.float32))


@pytest.mark.parametrize("prec,tol", [(O.BF16, 2.0 ** -7), (O.E4M3, 2.0 ** -2)])
def test_mxp_factors_accuracy_dd(prec, tol):
    n = 512
    A, b = O.generate(n, 9, dd=True)
    W, info = O.mxp_getrf(A, 128, prec)
    L = np.tril(W.astype(np.float64), -1) + np.eye(n)
    U = np.triu(W.astype(np.float64))
    rel = np.linalg.norm(L @ U - A) / np.linalg.norm(A)
    assert info == 0 and rel < tol
    # the FP32 solve with these factors is a usable preconditioner
    x = O.mxp_getrs(W, b)
    xr = np.linalg.solve(A, b)
    assert np.max(np.abs(x - xr)) / np.max(np.abs(xr)) < 8 * tol


# bar of the panel-by-panel comparison of the GPU's mixed-precision factors
# with the oracle replaying the GPU's quantized panels (tests/test_gpu_mxp.py)
from tests.mxp_compare import MXP_PANEL_BAR, panel_ratios, worst  # noqa: E402


@pytest.mark.parametrize("prec", [O.BF16, O.E4M3], ids=["bf16", "e4m3"])
def test_mxp_replay_of_own_factors_is_exact_and_a_planted_error_is_caught(prec):
    n, nb = 1024, 256
    A, _ = O.generate(n, 7, dd=True)
    W1, info = O.mxp_getrf(A, nb, prec)
    assert info == 0
    # replaying its own factors quantizes the same values: bitwise the same run
    W2, _ = O.mxp_getrf(A, nb, prec, replay=W1)
    assert np.array_equal(W1, W2)
    # a relative error of 1e-5 planted in one panel's product L21 = A21 U11^-1
    # exceeds the bar of the panel comparison, in that panel's L21
    for panel in (0, 2):
        W3, _ = O.mxp_getrf(A, nb, prec, replay=W1, plant=(panel, 1e-5))
        r, p, name = worst(panel_ratios(W3, W1, nb))
        assert (p, name) == (panel, "L21") and r > MXP_PANEL_BAR, (r, p, name)
