"""Pins of the oracle's decomposition (Sec. 3.1), Algorithms 1-2 (off-diagonal
closed forms) and Algorithm 3 (the level chain).

The chain is pinned by flows whose every step has a closed form: diagonal
shears sin(m (x1 + x2)) as the diagonal bands (exact discrete corrector) and
x2-shears as the off-diagonal part (exact line variance), so the composition
K_off -> K* -> K*_net -> K of Algorithm 3 can be written out by hand.
"""
import math

import numpy as np
import pytest

import inputs
from inputs import flows
import oracle


def test_decomposition_partitions_the_spectrum():
    spec = flows.continuous_spectrum(64, seed=7)
    edges = [1, 2, 4, 8, 16, 32, 65]
    lev, kind = oracle.band_of(spec, edges)
    assert np.all(lev >= 1) and np.all(kind >= 0)
    a, b = np.abs(spec.k1), np.abs(spec.k2)
    def level(m):
        return np.searchsorted(np.array(edges[1:]), m, side="right") + 1
    la, lb = level(a), level(b)
    # diagonal: both magnitudes in the same band; 12: |k1| band below |k2| band
    assert np.array_equal(kind == 0, la == lb)
    assert np.array_equal(kind == 1, la < lb)
    assert np.array_equal(kind == 2, la > lb)
    assert np.array_equal(lev, np.minimum(la, lb))
    # Hermitian partners land in the same part
    key = {(int(x), int(y)): (l, k) for x, y, l, k in zip(spec.k1, spec.k2, lev, kind)}
    for (x, y), v in key.items():
        assert key[(-x, -y)] == v


def test_bands_sum_to_the_field():
    spec = flows.continuous_spectrum(32, seed=3)
    edges = [1, 2, 4, 8, 16, 33]
    lev, kind = oracle.band_of(spec, edges)
    Nl, n = 64, 8
    total = oracle.patch_psi(spec, Nl, 5, 9, n)
    acc = np.zeros_like(total)
    for l in range(1, len(edges)):
        for k in (0, 1, 2):
            acc += oracle.patch_psi(spec, Nl, 5, 9, n, use=(lev == l) & (kind == k))
    np.testing.assert_allclose(acc, total, atol=1e-13)


def test_paper_two_level_example_parts():
    # Sec. 4.3 structure with alpha = 5 read as edges {1, 6, 51}: phi_c(5,5) -> psi_11,
    # phi_c(5,45) -> psi_12, phi_c(45,5) -> psi_21, phi_c(50,50) -> psi_22
    d = {}
    for (m1, m2) in [(5, 5), (5, 45), (45, 5), (50, 50)]:
        flows._add_sinsin(d, 0.2, m1, m2)
    spec = flows._from_dict(d)
    lev, kind = oracle.band_of(spec, [1, 6, 51])
    got = {(abs(int(a)), abs(int(b))): (int(l), int(k)) for a, b, l, k in zip(spec.k1, spec.k2, lev, kind)}
    assert got[(5, 5)] == (1, 0)
    assert got[(5, 45)] == (1, 1)
    assert got[(45, 5)] == (1, 2)
    assert got[(50, 50)] == (2, 0)


def test_patch_origin_snaps_to_nearest_lattice_node():
    # macro node i at i * 2 pi / N; lattice spacing 2 pi / Nl; ties round up
    assert oracle.patch_origin(3, 128, 64, 64) == 2 - 32   # 1.5 -> 2
    assert oracle.patch_origin(4, 128, 64, 64) == 2 - 32
    assert oracle.patch_origin(5, 32, 256, 32) == 40 - 16
    assert oracle.patch_origin(0, 32, 256, 32) == -16


@pytest.mark.parametrize("A,m", [(0.5, 8), (1.2, 20)])
def test_alg1_on_pure_x2_shear_equals_closed_form(A, m):
    # P7: psi_12 = A sin(m x2) is x1-independent, so every column gives
    # K*11 = B11 + <psi^2> / B22 = B11 + A^2 / (2 B22) (Eq. shearhomoY) and the
    # harmonic mean of a constant is that constant.
    spec = flows.shear_x2(A, m)
    use = np.ones(spec.n_modes, bool)
    n, Nl = 16, 16
    q12, q21 = oracle.offdiag_q(spec, use, ~use, Nl, 3, -4, n, 2 * math.pi)
    np.testing.assert_allclose(q12, A * A / 2, rtol=1e-13)
    assert not np.any(q21)
    B = np.array([0.3, 0.05, 0.7])
    np.testing.assert_allclose(oracle.offdiag_apply(q12, None, B),
                               [B[0] + A * A / (2 * B[2]), B[1], B[2]], rtol=1e-14)


def test_alg1_harmonic_mean_across_columns():
    # psi_12 = A cos(x1) sin(m x2): q(x1) = A^2 cos^2(x1) / 2, so
    # K11 = (mean_a 1 / (B11 + A^2 cos^2(x_a) / (2 B22)))^-1, which for a full period
    # equals the layered-medium value sqrt(a (a + b)), a = B11, b = A^2 / (2 B22)
    # ((1/2pi) int dx / (a + b cos^2 x) = 1 / sqrt(a (a + b))).
    A, m = 0.8, 12
    d = {}
    # cos(x1) sin(m x2) = [sin(m x2 + x1) + sin(m x2 - x1)] / 2
    for k1 in (1, -1):
        flows._add(d, (k1, m), -0.25j * A)
        flows._add(d, (-k1, -m), 0.25j * A)
    spec = flows._from_dict(d)
    use = np.ones(spec.n_modes, bool)
    n, Nl = 96, 96     # the column mean of this trig rational converges geometrically in n
    q12, _ = oracle.offdiag_q(spec, use, ~use, Nl, 0, 0, n, 2 * math.pi)
    xa = 2 * math.pi * np.arange(n) / Nl
    np.testing.assert_allclose(q12, A * A * np.cos(xa) ** 2 / 2, atol=1e-14)
    B = np.array([0.2, 0.0, 0.5])
    K = oracle.offdiag_apply(q12, None, B)
    a, b = B[0], A * A / (2 * B[2])
    assert K[0] == pytest.approx(math.sqrt(a * (a + b)), rel=1e-12)
    assert K[2] == B[2]


def test_alg2_one_zero_part_returns_the_other():
    rng = np.random.default_rng(0)
    q = rng.uniform(0.1, 0.5, 8)
    B = np.array([0.3, 0.02, 0.4])
    K = oracle.offdiag_apply(q, None, B)
    K2 = oracle.offdiag_apply(None, q, B)
    # an absent part leaves its component exactly; a zero-variance part gives the
    # harmonic mean of a constant line, i.e. that constant to rounding
    assert K[2] == B[2] and K[1] == B[1]
    assert K2[0] == B[0] and K2[1] == B[1]
    Kz = oracle.offdiag_apply(q, np.zeros(8), B)
    assert Kz[2] == pytest.approx(B[2], rel=1e-15)
    assert np.array_equal(oracle.offdiag_apply(None, None, B), B)
    both = oracle.offdiag_apply(q, q, B)
    np.testing.assert_allclose(both, [K[0], B[1], K2[2]], rtol=1e-15)


def _diag_shear_K(B, A, m, h, dt, nb, na):
    """Closed form of K[A sin(m(x1+x2)), B] on a periodic patch of spacing h."""
    mu = (4 * (B[0] + B[2]) * math.sin(m * h / 2) ** 2 + 2 * B[1] * math.sin(m * h) ** 2) / h ** 2
    sig = A * math.sin(m * h) / h
    z = dt * mu
    g = 1 - z + z * z / 2
    T = g ** (nb + 1) * (1 - g ** na) / ((1 - g) * na)
    e = sig ** 2 / (2 * mu) * (1 - T)
    return np.array([B[0] + e, B[1] - e, B[2] + e])


def test_alg3_chain_closed_form():
    # Two diagonal bands (diag shears at k = (1,1) and (4,4)) plus an off-diagonal
    # x2-shear (0, 8) (|k1| in level 1, |k2| in level 2 -> psi_12 of level 1).
    # Algorithm 3: Koff = K[psi_12; kappa] = kappa + A3^2/(2 kappa) in the 11 entry,
    # K* = K[psi_22; Koff], K*_net = K* - Koff + kappa I,
    # K = K[psi_11; K_off,1(K*_net)].
    A1, A2, A3, kappa = 0.6, 0.35, 0.3, 0.05
    spec = flows.combine(flows.shear_diag(A1, 1), flows.shear_diag(A2, 4), flows.shear_x2(A3, 8))
    edges = [1, 4, 16]
    n, N = 16, 4
    cfl, nb, na = 0.2, 300, 200
    nodes = [(0, 0), (1, 2), (3, 1)]
    K = oracle.chain(spec, edges, [n, n], N, kappa, nodes, cfl=cfl, n_burn_fixed=nb, n_avg_fixed=na)

    kI = np.array([kappa, 0.0, kappa])
    def koff(B):                       # Algorithm 1-2 with q12 = A3^2 / 2 on every column
        return np.array([B[0] + A3 ** 2 / (2 * B[2]), B[1], B[2]])
    def solve(B, A, m, h):
        sig = A * math.sin(m * h) / h
        dt = oracle.micro_dt(h, 2 * sig, B, cfl)       # max(|v1| + |v2|) = 2 sig on the patch
        return _diag_shear_K(B, A, m, h, dt, nb, na)
    h1, h2 = 2 * math.pi / n, 2 * math.pi / (4 * n)
    Koff1 = koff(kI)
    Kstar2 = solve(Koff1, A2, 4, h2)          # level 2 has no off-diagonal part
    Knet = Kstar2 - Koff1 + kI
    want = solve(koff(Knet), A1, 1, h1)
    for k in K:
        np.testing.assert_allclose(k, want, rtol=1e-11)


def test_prop1_parallel_shears_iterate_exactly():
    # Prop. 1: for L2-orthogonal parallel shears, one patch with both equals the
    # iterated homogenization, here discretely with the grid factors cos^2(m h / 2).
    A1, m1, A2, m2 = 0.5, 1, 0.3, 4
    B = np.array([0.2, 0.0, 0.1])
    n = 32
    h1, h2 = 2 * math.pi / n, 2 * math.pi / (4 * n)
    dt, nb, na = 0.05, 6000, 2000
    both = oracle.patch_k(oracle.patch_psi(flows.combine(flows.shear_x1(A1, m1), flows.shear_x1(A2, m2)),
                                           n, 0, 0, n), h1, B, dt, nb, na)
    fine = oracle.patch_k(oracle.patch_psi(flows.shear_x1(A2, m2), 4 * n, 0, 0, n), h2, B, 0.003, 60000, 2000)
    it = oracle.patch_k(oracle.patch_psi(flows.shear_x1(A1, m1), n, 0, 0, n), h1, fine, dt, nb, na)
    c = lambda m, h: math.cos(m * h / 2) ** 2
    exact_both = B[2] + (A1 ** 2 * c(m1, h1) + A2 ** 2 * c(m2, h1)) / (2 * B[0])
    exact_it = B[2] + (A1 ** 2 * c(m1, h1) + A2 ** 2 * c(m2, h2)) / (2 * B[0])
    assert both[2] == pytest.approx(exact_both, rel=1e-10)
    assert it[2] == pytest.approx(exact_it, rel=1e-10)
    # and both agree with the continuum value of Prop. 1 to the grid factors
    assert it[2] == pytest.approx(B[2] + (A1 ** 2 + A2 ** 2) / (2 * B[0]), rel=1e-2)


def test_translation_invariance_config_like():
    # P10: on a band periodic on the patch, every macro node's patch is a lattice
    # shift of the others, so the chain gives the same K everywhere
    spec = flows.cellular_hierarchy(2, 4)
    nodes = [(0, 0), (3, 5), (7, 2)]
    K = oracle.chain(spec, [1, 4, 16], [16, 16], 8, 0.05, nodes, n_burn_fixed=200, n_avg_fixed=100)
    np.testing.assert_allclose(K, np.repeat(K[:1], 3, 0), rtol=1e-12, atol=1e-14)
    assert abs(K[0, 0] - K[0, 2]) < 1e-12 * K[0, 0] and abs(K[0, 1]) < 1e-12
