"""Pins of the oracle's macro solver (Eq. homo) and direct simulation (Eq. model).

The macro scheme with constant K multiplies every Fourier mode by exactly
1 + z + z^2/2 per Heun step, z = -dt [4 K11 sin^2(t1/2) + 4 K22 sin^2(t2/2)
+ 2 K12 sin t1 sin t2] / H^2; the flux form conserves sum(U) for any K field.
"""
import math

import numpy as np
import pytest

from inputs import flows
import oracle


@pytest.mark.parametrize("p1,p2", [(1, 0), (2, 3), (5, -4)])
def test_macro_fourier_amplification(p1, p2):
    N = 16
    H = 2 * math.pi / N
    K = np.tile(np.array([0.3, 0.11, 0.2]), (N * N, 1))
    i = np.arange(N)
    U0 = np.cos(2 * math.pi * (p1 * i[None, :] + p2 * i[:, None]) / N)
    dt, ns = 0.01, 40
    U, mass = oracle.macro_run(U0, K, dt, ns)
    t1, t2 = 2 * math.pi * p1 / N, 2 * math.pi * p2 / N
    z = -dt * (4 * K[0, 0] * math.sin(t1 / 2) ** 2 + 4 * K[0, 2] * math.sin(t2 / 2) ** 2
               + 2 * K[0, 1] * math.sin(t1) * math.sin(t2)) / H ** 2
    np.testing.assert_allclose(U, U0 * (1 + z + z * z / 2) ** ns, atol=1e-13)


def test_macro_conserves_mass_with_variable_K():
    N = 32
    rng = np.random.default_rng(1)
    a = rng.uniform(0.1, 1.0, (N * N, 2))
    c = rng.uniform(-0.3, 0.3, N * N) * np.sqrt(a[:, 0] * a[:, 1])
    K = np.stack([a[:, 0], c, a[:, 1]], 1)
    U0 = flows.gaussian_u0(N)
    dt = oracle.macro_dt(K, N, 0.2)
    U, mass = oracle.macro_run(U0, K, dt, 200)
    assert np.max(np.abs(mass - mass[0])) < 1e-12 * mass[0]
    assert U.max() < U0.max()


def test_macro_dt_rule():
    N = 8
    K = np.tile([0.5, -0.2, 0.25], (N * N, 1))
    H = 2 * math.pi / N
    assert oracle.macro_dt(K, N, 0.2) == pytest.approx(0.2 * H * H / 0.95)


def test_dns_without_flow_matches_macro_with_kappa():
    # v = 0: the DNS operator is kappa times the 5-point Laplacian, the same
    # operator as the macro scheme with K = kappa I (two separate codes)
    N, kappa = 32, 0.3
    psi = np.zeros((N, N))
    U0 = flows.gaussian_u0(N)
    dt, ns = 0.02, 50
    u = oracle.dns_run(psi, kappa, dt, ns, U0)
    U, _ = oracle.macro_run(U0, np.tile([kappa, 0.0, kappa], (N * N, 1)), dt, ns)
    np.testing.assert_allclose(u, U, atol=1e-14)


def test_dns_fourier_mode_and_conservation():
    N, kappa = 64, 0.05
    spec = flows.cellular_two_scale(1.0, 0.3, 4)
    psi = oracle.grid_psi(spec, N)
    # psi on the grid equals the closed form
    x = 2 * math.pi * np.arange(N) / N
    ref = np.sin(x)[None, :] * np.sin(x)[:, None] + 0.3 * np.sin(4 * x)[None, :] * np.sin(4 * x)[:, None]
    np.testing.assert_allclose(psi, ref, atol=1e-13)
    u0 = flows.gaussian_u0(N)
    u = oracle.dns_run(psi, kappa, 0.005, 100, u0)
    h = 2 * math.pi / N
    assert abs(u.sum() - u0.sum()) < 1e-12 * u0.sum()
    Uc, m = oracle.coarse_grain(u, 16)
    assert m == pytest.approx(u.sum() * h * h, rel=1e-14)
    assert Uc.sum() * (2 * math.pi / 16) ** 2 == pytest.approx(m, rel=1e-12)


def _dns_shear_closed_form(A, m, N, dt, s, along):
    """Exact discrete solution of the DNS scheme with kappa = 0 for a shear and
    a single cosine across it (Eq. model with Heun's RK2, central differences).

    along = 1: psi = A sin(m x1), so v = (0, v2(x1)) with the central
    difference v2 = A cos(m x1) sin(m h)/h; u0 = cos(x2).  Each column x1 = x_a
    is advected on its own: D0y e^{i x2} = i sin(h)/h e^{i x2}, so the complex
    amplitude of e^{i x2} on column a is multiplied per step by
    g = 1 + z + z^2/2 with z = i dt v2(x_a) sin(h)/h, and u = Re(g^s e^{i x2}).
    along = 2 is the mirror: psi = A sin(m x2), v1 = -A cos(m x2) sin(m h)/h,
    u0 = cos(x1)."""
    h = 2 * math.pi / N
    x = h * np.arange(N)
    if along == 1:
        vel = A * np.cos(m * x) * math.sin(m * h) / h        # v2 on column a
    else:
        vel = -A * np.cos(m * x) * math.sin(m * h) / h       # v1 on row b
    z = 1j * dt * vel * math.sin(h) / h
    g = (1 + z + z * z / 2) ** s
    if along == 1:
        return np.real(g[None, :] * np.exp(1j * x)[:, None])  # [b][a]
    return np.real(g[:, None] * np.exp(1j * x)[None, :])


@pytest.mark.parametrize("along", [1, 2])
def test_dns_advection_of_a_shear_closed_form(along):
    # pins the sign and the orientation of the advection term v.grad u of the
    # direct simulation: a flipped sign conjugates g (the phase runs the other
    # way) and swapped components leave u0 unchanged
    N, A, m, dt, s = 32, 0.7, 3, 0.01, 150
    spec = flows.shear_x1(A, m) if along == 1 else flows.shear_x2(A, m)
    psi = oracle.grid_psi(spec, N)
    x = 2 * math.pi * np.arange(N) / N
    u0 = np.cos(x)[:, None] * np.ones(N)[None, :] if along == 1 else \
        np.ones(N)[:, None] * np.cos(x)[None, :]
    u = oracle.dns_run(psi, 0.0, dt, s, u0)
    want = _dns_shear_closed_form(A, m, N, dt, s, along)
    # the transport moved the field well away from u0
    assert np.abs(want - u0).max() > 0.5
    np.testing.assert_allclose(u, want, atol=1e-12)


def test_dns_shear_does_not_advect_along_itself():
    # psi = A sin(m x1) moves nothing along x1: u0 = cos(p x1) only diffuses,
    # with the 5-point amplification 1 + z + z^2/2, z = -4 dt kappa sin^2(p h/2)/h^2
    N, A, m, p, kappa, dt, s = 32, 0.7, 3, 2, 0.05, 0.01, 200
    h = 2 * math.pi / N
    psi = oracle.grid_psi(flows.shear_x1(A, m), N)
    x = h * np.arange(N)
    u0 = np.ones(N)[:, None] * np.cos(p * x)[None, :]
    u = oracle.dns_run(psi, kappa, dt, s, u0)
    z = -4 * dt * kappa * math.sin(p * h / 2) ** 2 / h ** 2
    np.testing.assert_allclose(u, u0 * (1 + z + z * z / 2) ** s, atol=1e-13)
