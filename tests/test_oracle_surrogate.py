"""Pins of the oracle's surrogate pieces: the patch features are a plain DFT
(checked against numpy's FFT); the second-order estimate Q they carry equals
the discrete shear closed form and the patch solve's K - B for shear flows,
and the patch solve's K - B to O(Pe^4) for a general flow; the MLP gradient
against central finite differences in FP64."""
import math

import numpy as np
import pytest

from inputs import flows
import oracle


def test_features_are_the_normalised_dft():
    n = 32
    rng = np.random.default_rng(0)
    psi = rng.standard_normal((n, n))
    psi -= psi.mean()
    B = np.array([0.3, 0.05, 0.5])
    f = oracle.features(psi, B, 0.01)
    assert f.shape == (585,)
    F = np.fft.fft2(psi) / n ** 2            # F[k2][k1] = n^-2 sum psi[b][a] e^{-2pi i(k1 a + k2 b)/n}
    want = []
    for k2 in range(-8, 9):
        for k1 in range(-8, 9):
            c = F[k2 % n, k1 % n] * 32.0 / (0.5 * (B[0] + B[2]))
            want += [c.real, c.imag]
    np.testing.assert_allclose(f[:578], want, atol=1e-11)
    np.testing.assert_allclose(f[578:582], [30.0, 5.0, 50.0, math.log(0.01)], rtol=1e-14)


def test_features_of_a_single_mode():
    # psi = cos(2 pi (2a + 3b)/n): the only nonzero coefficients are at +-(2, 3), value 1/2
    n = 32
    a = np.arange(n)
    psi = np.cos(2 * math.pi * (2 * a[None, :] + 3 * a[:, None]) / n)
    f = oracle.features(psi, np.array([1.0, 0.0, 1.0]), 1.0)
    c = f[:578].reshape(17, 17, 2) / 32.0
    assert c[3 + 8, 2 + 8, 0] == pytest.approx(0.5, abs=1e-14)
    assert c[-3 + 8, -2 + 8, 0] == pytest.approx(0.5, abs=1e-14)
    c[3 + 8, 2 + 8, 0] = c[-3 + 8, -2 + 8, 0] = 0
    assert np.abs(c).max() < 1e-14


def _steady_K(psi, h, B):
    # the time-stepped patch estimator run long past its relaxation time
    v1, v2 = oracle.velocity(psi, h)
    vmax = float(np.max(np.abs(v1) + np.abs(v2)))
    dt = oracle.micro_dt(h, vmax, B, 0.2)
    nb, na = oracle.micro_steps(2 * math.pi, B, dt, 40.0, 4.0)
    return oracle.patch_k(psi, h, B, dt, nb, na)


@pytest.mark.parametrize("k,axis", [(3, 1), (5, 2), (1, 1)])
def test_second_order_estimate_is_exact_for_shears(k, axis):
    # psi = a cos(2 pi k x_axis / n): the corrector of a shear solves a linear
    # equation with no advection of w, so the first-order solution is exact;
    # K_jj - B_jj = (a^2 / 2) cos^2(t/2) / B_ii (t = 2 pi k / n, i the shear
    # direction, j the other), and the patch solve gives the same.
    n, a = 24, 0.07
    idx = np.arange(n)
    line = a * np.cos(2 * math.pi * k * idx / n)
    psi = line[None, :].repeat(n, 0) if axis == 1 else line[:, None].repeat(n, 1)
    B = np.array([0.031, 0.009, 0.022])
    f = oracle.features(psi, B, 0.01)
    Q = oracle.second_order_K(f, B)
    t = 2 * math.pi * k / n
    if axis == 1:
        want = np.array([0.0, 0.0, 0.5 * a * a * math.cos(t / 2) ** 2 / B[0]])
    else:
        want = np.array([0.5 * a * a * math.cos(t / 2) ** 2 / B[2], 0.0, 0.0])
    np.testing.assert_allclose(Q, want, rtol=1e-12, atol=1e-15)
    h = 2 * math.pi / n
    K = _steady_K(psi, h, B)
    np.testing.assert_allclose(K - B, want, rtol=1e-8, atol=1e-13)


def test_second_order_estimate_is_the_small_peclet_limit():
    # a non-shear flow inside the 17 x 17 window with a full-tensor base: the
    # patch solve's K - B equals Q up to O(Pe^4), so halving the amplitude
    # shrinks the relative gap about fourfold (a wrong sign on the cross terms
    # of M or D would leave an O(1) gap)
    n = 20
    idx = np.arange(n)
    A, Bi = np.meshgrid(idx, idx)             # A: a (fast, x1), Bi: b (slow, x2)
    shape = (np.cos(2 * math.pi * (2 * A + 3 * Bi) / n) + 0.5 * np.sin(2 * math.pi * (A - 2 * Bi) / n)
             + 0.3 * np.cos(2 * math.pi * 4 * A / n))
    B = np.array([0.05, 0.012, 0.035])
    h = 2 * math.pi / n
    gaps = []
    for eps in (4e-3, 2e-3):
        psi = eps * shape
        Q = oracle.second_order_K(oracle.features(psi, B, 0.01), B)
        K = _steady_K(psi, h, B)
        gaps.append(np.linalg.norm(K - B - Q) / np.linalg.norm(Q))
        assert abs(Q[1]) > 0.05 * abs(Q[0])       # the cross term is exercised
    assert gaps[0] < 2e-2
    assert 3.0 < gaps[0] / gaps[1] < 5.0, gaps


def _params(d0, h, rng):
    return rng.uniform(-1, 1, oracle.mlp_param_count(d0, h)) * 0.3


def test_mlp_gradient_matches_finite_differences():
    rng = np.random.default_rng(1)
    d0, h, M = 7, 6, 5
    X = rng.standard_normal((M, d0))
    Y = rng.standard_normal((M, 3)) * 0.1
    p = _params(d0, h, rng)
    _, loss, g = oracle.mlp(X, p, h, bf16=False, Y=Y, want_grad=True)
    eps = 1e-6
    for q in rng.choice(p.size, 40, replace=False):
        pp = p.copy(); pp[q] += eps
        pm = p.copy(); pm[q] -= eps
        fd = (oracle.mlp(X, pp, h, bf16=False, Y=Y)[1] - oracle.mlp(X, pm, h, bf16=False, Y=Y)[1]) / (2 * eps)
        assert abs(fd - g[q]) <= 1e-6 * max(1e-3, abs(g[q])), (q, fd, g[q])


def test_mlp_forward_is_a_plain_network():
    # explicit numpy forward of the same network (exact-erf GELU), no bf16
    from math import erf
    rng = np.random.default_rng(2)
    d0, h, M = 5, 4, 3
    X = rng.standard_normal((M, d0))
    p = _params(d0, h, rng)
    o = 0
    layers = []
    for din, dout in [(d0, h), (h, h), (h, h), (h, 3)]:
        W = p[o:o + dout * din].reshape(dout, din); o += dout * din
        b = p[o:o + dout]; o += dout
        layers.append((W, b))
    a = X
    g = np.vectorize(lambda z: 0.5 * z * (1 + erf(z / math.sqrt(2))))
    for i, (W, b) in enumerate(layers):
        a = a @ W.T + b
        if i < 3:
            a = g(a)
    np.testing.assert_allclose(oracle.mlp(X, p, h, bf16=False), a, rtol=1e-13, atol=1e-15)


def test_bf16_emulation_rounds_like_bfloat16():
    import torch
    rng = np.random.default_rng(3)
    d0, h = 4, 4
    # identity-like net: check that inputs are rounded exactly as torch.bfloat16 rounds
    X = rng.standard_normal((2, d0)) * 1.234567
    p = np.zeros(oracle.mlp_param_count(d0, h))
    out32 = oracle.mlp(X, p, h, bf16=True)
    assert np.all(out32 == 0)
    xr = torch.tensor(X, dtype=torch.float32).to(torch.bfloat16).double().numpy()
    # one-layer probe: W1 = e_0 picks x_0; the result passes GELU and rounding
    p1 = p.copy(); p1[0] = 1.0
    o = h * d0 + h + 2 * (h * h + h)
    p1[o] = 1.0                               # W4[0][0]
    # W2 and W3 identity on unit 0
    p1[h * d0 + h] = 1.0
    p1[h * d0 + h + h * h + h] = 1.0
    from math import erf
    gl = lambda z: 0.5 * z * (1 + erf(z / math.sqrt(2)))
    bf = lambda v: float(torch.tensor(v, dtype=torch.float32).to(torch.bfloat16).double())
    want = [bf(gl(bf(gl(bf(gl(xr[m, 0])))))) for m in range(2)]
    np.testing.assert_allclose(oracle.mlp(X, p1, h, bf16=True)[:, 0], want, rtol=1e-15)


def _smooth_psi(n, rng, modes=6):
    a, b = np.meshgrid(np.arange(n), np.arange(n))
    psi = np.zeros((n, n))
    for _ in range(modes):
        k1, k2 = rng.integers(-3, 4, 2)
        ph = rng.uniform(0, 2 * math.pi)
        psi += rng.normal() * np.cos(2 * math.pi * (k1 * a + k2 * b) / n + ph)
    return psi - psi.mean()


@pytest.mark.parametrize("g", range(1, 8))
def test_patch_problem_is_equivariant_under_the_square_group(g):
    # the discrete corrector problem (central differences, periodic wrap, Heun,
    # window average) maps onto itself: the patch psi' = -psi o R^-1 (det R = -1)
    # or psi o R^-1 with base R B R^T has K' = R K R^T, to rounding
    from tests._parity import square_symmetry_psi, square_symmetry_tensor
    rng = np.random.default_rng(g)
    n = 16
    h = 2 * math.pi / n
    psi = 0.3 * _smooth_psi(n, rng)
    B = np.array([0.05, 0.012, 0.03])
    v1, v2 = oracle.velocity(psi, h)
    dt = oracle.micro_dt(h, float(np.max(np.abs(v1) + np.abs(v2))), B, 0.2)
    K = oracle.patch_k(psi, h, B, dt, 150, 100)
    psi_g = square_symmetry_psi(psi, g)
    B_g = square_symmetry_tensor(B, g)
    w1, w2 = oracle.velocity(psi_g, h)
    assert np.max(np.abs(w1) + np.abs(w2)) == pytest.approx(np.max(np.abs(v1) + np.abs(v2)), rel=1e-14)
    K_g = oracle.patch_k(psi_g, h, B_g, dt, 150, 100)
    want = square_symmetry_tensor(K, g)
    np.testing.assert_allclose(K_g, want, rtol=0, atol=1e-12 * np.abs(K).max())
    assert np.abs(psi_g - psi).max() > 0.1 * np.abs(psi).max()   # a different patch


def _feature_rule(f, g):
    # the signed permutation of a feature row that mlsd.h states for element g
    from tests._parity import square_symmetry_tensor
    out = np.array(f, dtype=np.float64)
    sign = -1.0 if bin(g).count("1") % 2 else 1.0
    for k2 in range(-8, 9):
        for k1 in range(-8, 9):
            q1, q2 = (k2, k1) if g & 4 else (k1, k2)
            s1 = -q1 if g & 1 else q1
            s2 = -q2 if g & 2 else q2
            d = 2 * ((k2 + 8) * 17 + k1 + 8)
            s = 2 * ((s2 + 8) * 17 + s1 + 8)
            out[d:d + 2] = sign * np.asarray(f)[s:s + 2]
    out[578:581] = square_symmetry_tensor(f[578:581], g)
    out[582:585] = square_symmetry_tensor(f[582:585], g)
    return out


@pytest.mark.parametrize("g", range(1, 8))
def test_features_of_the_mapped_patch_follow_the_stated_rule(g):
    # features of the mapped patch (DFT, base, second-order estimate) are the
    # signed permutation of the patch's own features
    from tests._parity import square_symmetry_psi, square_symmetry_tensor
    n, kappa = 32, 2e-3
    spec = flows.continuous_spectrum(40, seed=9)
    psi = oracle.patch_psi(spec, 96, 5, 17, n)
    B = np.array([3.0, 0.7, 2.0]) * kappa
    f = oracle.features(psi, B, kappa)
    f_g = oracle.features(square_symmetry_psi(psi, g), square_symmetry_tensor(B, g), kappa)
    scale = np.abs(f[:578]).max()
    np.testing.assert_allclose(f_g[:578], _feature_rule(f, g)[:578], rtol=0, atol=1e-12 * scale)
    np.testing.assert_allclose(f_g[578:], _feature_rule(f, g)[578:], rtol=1e-12, atol=1e-15)
