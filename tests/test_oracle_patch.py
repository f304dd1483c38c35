"""Pins of the oracle's patch solve K[psi, B; D] (HMM steps 1-3, Sec. 2.2).

Each test fixes the oracle against something other than itself: the discrete
closed form of shear flows (Eq. shearhomoX/Y with the second-order grid
factor), the exact geometric transient of Heun's method, a direct dense
solve of the steady corrector equation, the kappa-only limit, conservation,
symmetry, and the small-Peclet asymptotics of cellular flows.
"""
import math

import numpy as np
import pytest

import inputs
import oracle


def _patch(spec, n, Nl=None, ox=0, oy=0):
    Nl = n if Nl is None else Nl
    h = 2 * math.pi / Nl
    return oracle.patch_psi(spec, Nl, ox, oy, n), h


def _transient(z, n_burn, n_avg):
    """1/n_avg * sum_{s=n_burn+1}^{n_burn+n_avg} g^s, g = 1 - z + z^2/2 (Heun on c' = -lam c + sig)."""
    g = 1.0 - z + 0.5 * z * z
    return g ** (n_burn + 1) * (1.0 - g ** n_avg) / ((1.0 - g) * n_avg)


def test_kappa_only_limit_is_exact():
    # v = 0: every corrector stays 0 and K = B bit for bit (P1)
    n = 16
    psi = np.zeros((n, n))
    B = np.array([0.37, -0.11, 0.52])
    K, w = oracle.patch_k(psi, 0.3, B, 0.01, 50, 50, want_w=True)
    assert np.array_equal(K, B)
    assert not np.any(w)


@pytest.mark.parametrize("m,A,phase", [(3, 0.7, 0.0), (5, 1.3, 0.4), (1, 0.2, 1.1)])
@pytest.mark.parametrize("B", [(0.3, 0.0, 0.2), (0.3, 0.07, 0.2), (1.0, -0.3, 2.0)])
def test_shear_x1_discrete_closed_form(m, A, phase, B):
    # psi = A sin(m x1 + phase): v = (0, v2(x1)); with the second-order grid factor
    # K22 = B22 + A^2 cos^2(m h / 2) / (2 B11) (Eq. shearhomoX), K11 and K12 unchanged,
    # and Heun's transient is geometric with z = dt * 4 B11 sin^2(m h / 2) / h^2.
    n = 16
    psi, h = _patch(inputs.flows.shear_x1(A, m, phase), n)
    B = np.array(B)
    dt, nb, na = 0.02, 37, 53
    K = oracle.patch_k(psi, h, B, dt, nb, na)
    lam = 4 * B[0] * math.sin(m * h / 2) ** 2 / h ** 2
    enh = A ** 2 * math.cos(m * h / 2) ** 2 / (2 * B[0]) * (1 - _transient(dt * lam, nb, na))
    np.testing.assert_allclose(K, [B[0], B[1], B[2] + enh], rtol=1e-12, atol=1e-14)


@pytest.mark.parametrize("m,A", [(2, 0.9), (4, 0.3)])
def test_shear_x2_discrete_closed_form(m, A):
    # mirror: psi = A sin(m x2) -> K11 = B11 + A^2 cos^2(m h/2) / (2 B22) (Eq. shearhomoY)
    n = 16
    psi, h = _patch(inputs.flows.shear_x2(A, m), n)
    B = np.array([0.4, 0.1, 0.25])
    dt, nb, na = 0.02, 400, 300
    K = oracle.patch_k(psi, h, B, dt, nb, na)
    lam = 4 * B[2] * math.sin(m * h / 2) ** 2 / h ** 2
    enh = A ** 2 * math.cos(m * h / 2) ** 2 / (2 * B[2]) * (1 - _transient(dt * lam, nb, na))
    np.testing.assert_allclose(K, [B[0] + enh, B[1], B[2]], rtol=1e-12, atol=1e-14)


@pytest.mark.parametrize("B", [(0.3, 0.0, 0.3), (0.5, 0.12, 0.2), (0.5, -0.2, 0.4)])
def test_diagonal_shear_pins_cross_derivative(B):
    # psi = A sin(m (x1 + x2)): advection drops out (v1 = -v2, D0x w = D0y w) and the
    # corrector is c cos(m s) with decay rate
    #   mu = [4 (B11 + B22) sin^2(m h/2) + 2 B12 sin^2(m h)] / h^2,
    # so K = B + sig^2 / (2 mu) [[1, -1], [-1, 1]] (1 - transient), sig = A sin(m h) / h.
    # A wrong sign or factor on the mixed derivative, or swapped v components, fails here.
    n, m, A = 16, 3, 0.8
    psi, h = _patch(inputs.flows.shear_diag(A, m), n)
    B = np.array(B)
    mu = (4 * (B[0] + B[2]) * math.sin(m * h / 2) ** 2 + 2 * B[1] * math.sin(m * h) ** 2) / h ** 2
    sig = A * math.sin(m * h) / h
    dt, nb, na = 0.01, 120, 80
    K = oracle.patch_k(psi, h, B, dt, nb, na)
    e = sig ** 2 / (2 * mu) * (1 - _transient(dt * mu, nb, na))
    np.testing.assert_allclose(K, [B[0] + e, B[1] - e, B[2] + e], rtol=1e-12, atol=1e-14)


def _direct_steady_K(psi, h, B):
    """K from a dense direct solve of f_j(w) = 0 with sum(w) = 0 (tiny grids only)."""
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
        rhs = np.concatenate([-src, [0.0]])
        w = np.linalg.lstsq(A, rhs, rcond=None)[0]
        W.append(w.reshape(n, n))
    S = np.array([[np.mean(v * w) for w in W] for v in (v1, v2)])   # S[i][j] = <v_i w_j>
    return np.array([B[0] + S[0, 0], B[1] + 0.5 * (S[0, 1] + S[1, 0]), B[2] + S[1, 1]])


def test_time_stepping_converges_to_direct_steady_solve():
    # P5: the estimator after a long burn-in equals the steady corrector's flux
    n = 12
    spec = inputs.flows.combine(inputs.flows.cellular_two_scale(0.6, 0.25, 2),
                                inputs.flows.shear_x2(0.3, 3, 0.5))
    psi, h = _patch(spec, n)
    B = np.array([0.45, 0.08, 0.3])
    v1, v2 = oracle.velocity(psi, h)
    vmax = float(np.max(np.abs(v1) + np.abs(v2)))
    dt = oracle.micro_dt(h, vmax, B, 0.2)
    nb, na = oracle.micro_steps(2 * math.pi, B, dt, 40.0, 4.0)
    K = oracle.patch_k(psi, h, B, dt, nb, na)
    Kd = _direct_steady_K(psi, h, B)
    np.testing.assert_allclose(K, Kd, rtol=1e-10, atol=1e-12)
    # and the enhancement is positive semidefinite (P9)
    D = np.array([[K[0] - B[0], K[1] - B[1]], [K[1] - B[1], K[2] - B[2]]])
    assert np.linalg.eigvalsh(D).min() > -1e-12


def test_corrector_mean_is_conserved():
    # P4: sum_ab w_j stays 0 (discrete div v = 0 and a zero-mean source)
    n = 16
    spec = inputs.flows.cellular_two_scale(1.0, 0.5, 3)
    psi, h = _patch(spec, n)
    B = np.array([0.2, 0.03, 0.25])
    K, w = oracle.patch_k(psi, h, B, 0.005, 300, 10, want_w=True)
    assert abs(w[0].sum()) < 1e-12 * np.abs(w[0]).sum()
    assert abs(w[1].sum()) < 1e-12 * np.abs(w[1]).sum()
    assert np.abs(w).max() > 1e-3


def test_cellular_symmetry():
    # P9: sin x sin y is symmetric under x1 <-> x2 and odd under x1 -> -x1:
    # K11 = K22 and K12 = 0 (to rounding)
    n = 32
    psi, h = _patch(inputs.flows.cellular_two_scale(1.0, 0.0, 1), n)
    B = np.array([0.1, 0.0, 0.1])
    v1, v2 = oracle.velocity(psi, h)
    dt = oracle.micro_dt(h, float(np.max(np.abs(v1) + np.abs(v2))), B, 0.2)
    K = oracle.patch_k(psi, h, B, dt, 2000, 500)
    assert abs(K[0] - K[2]) < 1e-12 * K[0]
    assert abs(K[1]) < 1e-12 * K[0]
    assert K[0] > B[0]


def test_cellular_small_peclet_asymptotics():
    # psi = A sin x sin y at A/kappa = 0.05: K - kappa = A^2 cos^2(h/2) / (8 kappa) (1 + O(Pe^2))
    n, kappa = 32, 0.2
    A = 0.05 * kappa
    psi, h = _patch(inputs.flows.cellular_two_scale(A, 0.0, 1), n)
    B = np.array([kappa, 0.0, kappa])
    v1, v2 = oracle.velocity(psi, h)
    dt = oracle.micro_dt(h, float(np.max(np.abs(v1) + np.abs(v2))), B, 0.2)
    nb, na = oracle.micro_steps(2 * math.pi, B, dt, 16.0, 4.0)
    K = oracle.patch_k(psi, h, B, dt, nb, na)
    pred = A ** 2 * math.cos(h / 2) ** 2 / (8 * kappa)
    assert abs((K[0] - kappa) / pred - 1) < 5e-3


def test_micro_dt_and_window_rules():
    # G4 / G5 readings: CFL on advection and diffusion, tau = L^2 / (4 pi^2 lambda_min)
    B = np.array([0.02, 0.0, 0.01])
    h = 0.1
    assert oracle.lambda_min(B) == pytest.approx(0.01)
    dt = oracle.micro_dt(h, 2.0, B, 0.2)
    assert dt == pytest.approx(0.2 * min(h / 2.0, h * h / (2 * 0.03)))
    nb, na = oracle.micro_steps(2 * math.pi, B, dt, 8.0, 4.0)
    tau = 1.0 / 0.01
    assert nb == math.ceil(8 * tau / dt) and na == math.ceil(4 * tau / dt)
    # pure diffusion: only the diffusive bound
    assert oracle.micro_dt(h, 0.0, B, 0.2) == pytest.approx(0.2 * h * h / 0.06)


def _steady(psi, h, B, want_w=False):
    v1, v2 = oracle.velocity(psi, h)
    vmax = float(np.max(np.abs(v1) + np.abs(v2)))
    dt = oracle.micro_dt(h, vmax, B, 0.2)
    nb, na = oracle.micro_steps(2 * math.pi, B, dt, 40.0, 4.0)
    return oracle.patch_k(psi, h, B, dt, nb, na, want_w=want_w)


@pytest.mark.parametrize("flow", ["x1", "x2", "diag"])
def test_energy_form_is_exact_for_shears(flow):
    # for a shear the advection of w vanishes (w depends on the shear coordinate
    # only, and for the diagonal shear D0x w = D0y w against v1 = -v2), so summing
    # the steady corrector equation against w_k by parts gives E = K - B exactly;
    # the diagonal shear with B12 != 0 pins the mixed-derivative term's form
    n = 16
    spec = {"x1": inputs.flows.shear_x1(0.7, 3, 0.2), "x2": inputs.flows.shear_x2(0.5, 2),
            "diag": inputs.flows.shear_diag(0.6, 2)}[flow]
    psi, h = _patch(spec, n)
    B = np.array([0.4, 0.09, 0.25])
    K, w = _steady(psi, h, B, want_w=True)
    E, mass = oracle.corrector_energy(w, h, B)
    np.testing.assert_allclose(E, K - B, rtol=1e-9, atol=1e-13)
    assert np.abs(K - B).max() > 1e-2
    assert np.abs(mass).max() < 1e-13 * np.abs(w).max()


def test_energy_form_converges_to_flux_form():
    # for a general flow the central advection term is not skew-adjoint on the
    # grid, so E and K - B differ by the O(h^2) truncation: doubling n cuts the
    # gap about fourfold (a plain sum by parts would have made it vanish)
    spec = inputs.flows.combine(inputs.flows.cellular_two_scale(0.6, 0.25, 2),
                                inputs.flows.shear_x2(0.3, 3, 0.5))
    B = np.array([0.45, 0.08, 0.3])
    gaps = []
    for n in (16, 32):
        psi, h = _patch(spec, n)
        K, w = _steady(psi, h, B, want_w=True)
        E, _ = oracle.corrector_energy(w, h, B)
        gaps.append(np.linalg.norm(E - (K - B)) / np.linalg.norm(K - B))
    assert gaps[0] > 1e-4
    assert 3.0 < gaps[0] / gaps[1] < 5.0, gaps
