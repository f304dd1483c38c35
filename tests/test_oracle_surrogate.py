"""Pins of the oracle's surrogate pieces: the patch features are a plain DFT
(checked against numpy's FFT); the perturbation moments T_m of the steady
corrector equation they carry give the discrete shear closed form (T_2, with
every higher moment zero) and, summed, the dense direct solve of the steady
corrector for a general flow with a full-tensor base; the resummation (Wynn's
epsilon algorithm) reproduces the value of a rational function from its Taylor
coefficients (the defining property of the Pade approximant) and matches the
Pade approximant solved from its linear equations; the MLP gradient against
central finite differences in FP64."""
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
    assert f.shape == (606,)
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


def _direct_steady_K(psi, h, B):
    """K from a dense direct solve of the steady corrector f_j(w) = 0 with sum(w) = 0."""
    n = psi.shape[0]
    N = n * n
    v1, v2 = oracle.velocity(psi, h)
    W = []
    for j in (1, 2):
        src = oracle.corrector_rhs(psi, h, B, j, np.zeros((n, n))).ravel()
        M = np.zeros((N, N))
        for c in range(N):
            e = np.zeros(N); e[c] = 1.0
            M[:, c] = oracle.corrector_rhs(psi, h, B, j, e.reshape(n, n)).ravel() - src
        A = np.vstack([M, np.ones((1, N))])
        w = np.linalg.lstsq(A, np.concatenate([-src, [0.0]]), rcond=None)[0]
        W.append(w.reshape(n, n))
    S = np.array([[np.mean(v * w) for w in W] for v in (v1, v2)])
    return np.array([B[0] + S[0, 0], B[1] + 0.5 * (S[0, 1] + S[1, 0]), B[2] + S[1, 1]])


@pytest.mark.parametrize("k,axis", [(3, 1), (5, 2), (1, 1)])
def test_series_of_a_shear_is_its_closed_form(k, axis):
    # psi = a cos(2 pi k x_axis / n): the corrector of a shear is not advected
    # (A c = 0), so T_2 is exact and every higher moment vanishes;
    # K_jj - B_jj = (a^2 / 2) cos^2(t/2) / B_ii (t = 2 pi k / n, i the shear
    # direction, j the other), which the patch solve also gives
    n, a = 24, 0.07
    idx = np.arange(n)
    line = a * np.cos(2 * math.pi * k * idx / n)
    psi = line[None, :].repeat(n, 0) if axis == 1 else line[:, None].repeat(n, 1)
    B = np.array([0.031, 0.009, 0.022])
    T = oracle.series(psi, B)
    t = 2 * math.pi * k / n
    if axis == 1:
        want = np.array([0.0, 0.0, 0.5 * a * a * math.cos(t / 2) ** 2 / B[0]])
    else:
        want = np.array([0.5 * a * a * math.cos(t / 2) ** 2 / B[2], 0.0, 0.0])
    np.testing.assert_allclose(T[0], want, rtol=1e-12, atol=1e-15)
    assert np.abs(T[1:]).max() < 1e-13 * np.abs(want).max()
    P2, P3, E, gap = oracle.series_estimate(T)
    np.testing.assert_allclose(E, want, rtol=1e-12, atol=1e-15)
    assert gap < 1e-13 * np.abs(want).max()
    h = 2 * math.pi / n
    np.testing.assert_allclose(_steady_K(psi, h, B) - B, want, rtol=1e-8, atol=1e-13)


def _general_flow(n, eps):
    idx = np.arange(n)
    A, Bi = np.meshgrid(idx, idx)             # A: a (fast, x1), Bi: b (slow, x2)
    shape = (np.cos(2 * math.pi * (2 * A + 3 * Bi) / n) + 0.5 * np.sin(2 * math.pi * (A - 2 * Bi) / n)
             + 0.3 * np.cos(2 * math.pi * 4 * A / n))
    return eps * shape


def test_series_sums_to_the_direct_steady_solve():
    # the moments are the terms of the Neumann series of (L0 + A) w = -v_j: for
    # a small Peclet number, T_2 + ... + T_20 is the dense direct solve's K - B
    n = 12
    psi = _general_flow(n, 0.02)
    B = np.array([0.05, 0.012, 0.035])
    h = 2 * math.pi / n
    Kd = _direct_steady_K(psi, h, B)
    T = oracle.series(psi, B, M=20)
    assert abs(T[0, 1]) > 0.05 * abs(T[0, 0])          # the cross term is exercised
    assert np.abs(T[2]).max() > 1e-3 * np.abs(T[0]).max()  # so are the higher orders
    np.testing.assert_allclose(B + T.sum(0), Kd, rtol=0, atol=1e-12 * np.abs(Kd - B).max())


def test_series_truncation_error_has_the_right_order():
    # the partial sum T_2 + ... + T_6 misses the O(v^7) tail: halving the amplitude
    # shrinks the gap to the direct solve ~2^7-fold (a wrong T_4 would leave O(v^4))
    n = 12
    B = np.array([0.05, 0.012, 0.035])
    h = 2 * math.pi / n
    gaps = []
    for eps in (0.08, 0.04):
        psi = _general_flow(n, eps)
        Kd = _direct_steady_K(psi, h, B)
        S6 = oracle.series(psi, B, M=6).sum(0)
        gaps.append(np.abs(B + S6 - Kd).max())
    assert 60 < gaps[0] / gaps[1] < 300, gaps


def _taylor_of_rational(a, b, count):
    """Taylor coefficients of (a0 + a1 x + ...) / (1 + b1 x + ...) by series division."""
    c = np.zeros(count)
    for k in range(count):
        v = a[k] if k < len(a) else 0.0
        for j in range(1, min(k, len(b) - 1) + 1):
            v -= b[j] * c[k - j]
        c[k] = v
    return c


def test_wynn_reproduces_a_rational_function():
    # the [K/K] Pade approximant of a rational function of degree (K, K) is the
    # function itself: from its Taylor coefficients Wynn's epsilon gives f(1),
    # even where the Taylor series diverges at 1
    rng = np.random.default_rng(4)
    for K in (1, 2, 3, 4):
        for _ in range(3):
            a = rng.uniform(-1, 1, K + 1)
            # denominator prod_i (1 - x / r_i): poles at 0.35 <= |x| <= 0.9, so the
            # Taylor series at 0 diverges at x = 1
            roots = rng.uniform(0.35, 0.9, K) * rng.choice([-1.0, 1.0], K)
            b = np.poly(roots)[::-1]
            b = b / b[0]
            c = _taylor_of_rational(a, b, 2 * K + 1)
            T = np.zeros((4 * K + 2, 3))
            T[0::2, 0] = c                      # pair k = T_(2k+2) + T_(2k+3) = c_k
            f1 = np.polyval(a[::-1], 1.0) / np.polyval(b[::-1], 1.0)
            assert oracle.wynn(T, 0, K) == pytest.approx(f1, rel=1e-7, abs=1e-12)
    # a geometric series of ratio -3 (divergent at 1): [1/1] = 1 / (1 + 3), with the
    # terms split between the two moments of each pair
    T = np.zeros((6, 3))
    T[:, 1] = [0.25, 0.75, -1.0, -2.0, 4.5, 4.5]
    assert oracle.wynn(T, 1, 1) == pytest.approx(0.25, rel=1e-14)


def test_wynn_matches_the_pade_linear_system():
    # [K/K](1) = p(1) / q(1) with q_0 = 1, sum_j q_j c_(k-j) = 0 for k = K+1..2K and
    # p_k = sum_(j<=k) q_j c_(k-j) for k <= K: solved with numpy on random data
    rng = np.random.default_rng(5)
    for K in (2, 3, 4):
        c = rng.standard_normal(2 * K + 1) * 0.5 ** np.arange(2 * K + 1)
        A = np.array([[c[k - j] for j in range(1, K + 1)] for k in range(K + 1, 2 * K + 1)])
        q = np.concatenate([[1.0], np.linalg.solve(A, -c[K + 1:2 * K + 1])])
        p = [sum(q[j] * c[k - j] for j in range(k + 1)) for k in range(K + 1)]
        T = np.zeros((4 * K + 2, 3))
        w = rng.uniform(0, 1, 2 * K + 1)
        T[0::2, 2] = w * c                  # any split of c_k over the pair
        T[1::2, 2] = (1 - w) * c
        assert oracle.wynn(T, 2, K) == pytest.approx(sum(p) / sum(q), rel=1e-9)


def test_estimate_converges_where_the_series_diverges():
    # a general flow whose moments grow (|T_4 / T_2| ~ 0.8 at this amplitude): the
    # partial sums drift away from the dense direct solve, the [4/4] approximant
    # of the pair series lands on it
    n = 12
    B = np.array([0.05, 0.012, 0.035])
    h = 2 * math.pi / n
    psi = _general_flow(n, 0.16)
    Kd = _direct_steady_K(psi, h, B)
    T = oracle.series(psi, B)
    P2, P3, E, gap = oracle.series_estimate(T)
    assert np.abs(T[2]).max() > 0.5 * np.abs(T[0]).max()
    assert np.abs(B + T.sum(0) - Kd).max() > 0.1 * np.abs(Kd - B).max()
    assert np.abs(B + E - Kd).max() < 1e-3 * np.abs(Kd - B).max()
    assert np.abs(E - P3).max() == pytest.approx(gap, rel=1e-14)


def test_features_carry_the_series():
    n = 16
    psi = _general_flow(n, 0.05)
    B = np.array([0.05, 0.012, 0.035])
    f = oracle.features(psi, B, 0.01)
    T = oracle.series(psi, B)
    P2, P3, E, _ = oracle.series_estimate(T)
    sc = 10.0 / (B[0] + B[2])
    np.testing.assert_allclose(np.sinh(f[582:597]), sc * T[:5].ravel(), rtol=1e-12, atol=1e-300)
    np.testing.assert_allclose(np.sinh(f[597:600]), sc * P2, rtol=1e-12)
    np.testing.assert_allclose(np.sinh(f[600:603]), sc * P3, rtol=1e-12)
    np.testing.assert_allclose(np.sinh(f[603:606]), sc * E, rtol=1e-12)


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
    for q in range(582, 606, 3):              # T_2..T_6, [4/4], [6/6], [8/8]: tensors
        out[q:q + 3] = np.arcsinh(square_symmetry_tensor(np.sinh(np.asarray(f[q:q + 3])), g))
    return out


@pytest.mark.parametrize("g", range(1, 8))
def test_features_of_the_mapped_patch_follow_the_stated_rule(g):
    # features of the mapped patch (DFT, base, series moments) are the
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
    np.testing.assert_allclose(f_g[578:597], _feature_rule(f, g)[578:597], rtol=1e-12, atol=1e-15)
    # the resummed values (Wynn's epsilon) amplify the rounding of the moments
    np.testing.assert_allclose(f_g[597:], _feature_rule(f, g)[597:], rtol=1e-8, atol=1e-12)


@pytest.mark.parametrize("n", [128, 256])
def test_large_patch_features_are_the_full_resolution_dft_window(n):
    # a band resolved on the patch (local modes |k| <= 3) has the same DFT window on the
    # 64 x 64 sub-lattice as on all n x n nodes: the sub-lattice features equal the
    # window of the full-resolution transform (normalised by n^2)
    rng = np.random.default_rng(n)
    psi = _smooth_psi(n, rng)
    B = np.array([0.3, 0.05, 0.5])
    f = oracle.features(psi, B, 0.01)
    F = np.fft.fft2(psi) / n ** 2
    want = []
    for k2 in range(-8, 9):
        for k1 in range(-8, 9):
            c = F[k2 % n, k1 % n] * 32.0 / (0.5 * (B[0] + B[2]))
            want += [c.real, c.imag]
    np.testing.assert_allclose(f[:578], want, atol=1e-11)
    # and it is the 64 x 64 rule: the features of the samples every n/64-th node
    s = n // 64
    q = psi[::s, ::s] - psi[::s, ::s].mean()
    np.testing.assert_allclose(f, oracle.features(q, B, 0.01), rtol=1e-9, atol=1e-10)


def test_large_patch_moments_converge_with_the_grid():
    # the moments on the sub-lattice are the grid moments of a coarser resolution of the
    # same band: against the full 128 x 128 grid and 256 x 256 grid, T_2..T_6 differ by
    # the second-order truncation error, which falls ~4x from 64 to 128 nodes a side
    rng = np.random.default_rng(5)
    a, b = np.meshgrid(np.arange(256), np.arange(256))
    psi256 = np.zeros((256, 256))
    for _ in range(5):
        k1, k2 = rng.integers(-2, 3, 2)
        ph = rng.uniform(0, 2 * math.pi)
        psi256 += 0.02 * rng.normal() * np.cos(2 * math.pi * (k1 * a + k2 * b) / 256 + ph)
    psi256 -= psi256.mean()
    B = np.array([0.01, 0.002, 0.015])
    T = {m: oracle.series(psi256[::256 // m, ::256 // m], B, M=6) for m in (64, 128, 256)}
    f = oracle.features(psi256, B, 0.01)
    got = np.sinh(f[582:597]).reshape(5, 3) * (B[0] + B[2]) / 10.0
    np.testing.assert_allclose(got, T[64], rtol=1e-9, atol=1e-15)
    e64 = np.abs(T[64] - T[256]).max()
    e128 = np.abs(T[128] - T[256]).max()
    scale = np.abs(T[256]).max()
    assert e64 < 0.05 * scale
    assert 3.0 < e64 / e128 < 5.5, (e64, e128)
