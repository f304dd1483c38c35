"""Pins of the oracle's surrogate pieces: the patch features are a plain DFT
(checked against numpy's FFT), and the MLP gradient against central finite
differences in FP64."""
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
    F = np.fft.fft2(psi) / n ** 2            # F[k2][k1] = n^-2 sum psi[b][a] e^{-2pi i(k1 a + k2 b)/n}
    want = []
    for k2 in range(-8, 9):
        for k1 in range(-8, 9):
            c = F[k2 % n, k1 % n] / (0.5 * (B[0] + B[2]))
            want += [c.real, c.imag]
    np.testing.assert_allclose(f[:578], want, atol=1e-13)
    np.testing.assert_allclose(f[578:], [30.0, 5.0, 50.0, math.log(0.01)], rtol=1e-14)


def test_features_of_a_single_mode():
    # psi = cos(2 pi (2a + 3b)/n): the only nonzero coefficients are at +-(2, 3), value 1/2
    n = 32
    a = np.arange(n)
    psi = np.cos(2 * math.pi * (2 * a[None, :] + 3 * a[:, None]) / n)
    f = oracle.features(psi, np.array([1.0, 0.0, 1.0]), 1.0)
    c = f[:578].reshape(17, 17, 2)
    assert c[3 + 8, 2 + 8, 0] == pytest.approx(0.5, abs=1e-14)
    assert c[-3 + 8, -2 + 8, 0] == pytest.approx(0.5, abs=1e-14)
    c[3 + 8, 2 + 8, 0] = c[-3 + 8, -2 + 8, 0] = 0
    assert np.abs(c).max() < 1e-14


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
