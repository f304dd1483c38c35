"""Pins of the oracle's solvers with the Sec. 4 boundary conditions.

The paper's numerical examples solve on [0,1]^2 with u = 1 at x1 = 0, u = 0 at
x1 = 1, periodic in x2, from a step.  The library poses the same problem on
[0, 2 pi] x [0, 2 pi) (x -> 2 pi x, t -> 4 pi^2 t, v -> v / 2 pi, psi
unchanged): column 0 of the node grid is the boundary x1 = 0 and a virtual
column N the boundary x1 = 2 pi.  The pins:
  * discrete sine modes sin(pi p i / N) cos(q x2) are eigenvectors of the
    scheme with constant diagonal K and homogeneous boundaries, amplified per
    Heun step by 1 + z + z^2/2, z = -dt (4 K11 sin^2(pi p / 2N)
    + 4 K22 sin^2(q H / 2)) / H^2;
  * the linear profile between the boundary values is steady for any constant
    full-tensor K (the cross terms of an x2-independent field cancel);
  * an x2-independent field with K varying in x1 only follows a 1-D
    finite-difference scheme written out separately below;
  * the direct simulation with v = 0 is the macro scheme with K = kappa I,
    and with kappa = 0 and a shear v = (v1(x2), 0) every row is a 1-D central
    advection problem.
"""
import math

import numpy as np
import pytest

from inputs import flows
import oracle


def _heun_1d(u, rhs, dt, s):
    for _ in range(s):
        us = u + dt * rhs(u)
        u = 0.5 * (u + us + dt * rhs(us))
    return u


@pytest.mark.parametrize("p,q", [(1, 0), (3, 2), (7, 5)])
def test_sine_mode_amplification(p, q):
    N = 32
    H = 2 * math.pi / N
    K = np.tile([0.4, 0.0, 0.25], (N * N, 1))
    i, j = np.arange(N), np.arange(N)
    U0 = np.sin(math.pi * p * i / N)[None, :] * np.cos(q * H * j)[:, None]
    dt, s = 0.02, 60
    U = oracle.macro_run_dirichlet(U0, K, dt, s, 0.0, 0.0)
    z = -dt * (4 * 0.4 * math.sin(math.pi * p / (2 * N)) ** 2
               + 4 * 0.25 * math.sin(q * H / 2) ** 2) / H ** 2
    want = U0 * (1 + z + z * z / 2) ** s
    assert abs((1 + z + z * z / 2) ** s) < 0.9
    np.testing.assert_allclose(U, want, atol=1e-13)


def test_linear_profile_is_steady_with_cross_terms():
    N = 24
    K = np.tile([0.7, -0.3, 0.5], (N * N, 1))
    U0 = np.tile(1.0 - np.arange(N) / N, (N, 1))
    U = oracle.macro_run_dirichlet(U0, K, 0.01, 100, 1.0, 0.0)
    np.testing.assert_allclose(U, U0, atol=1e-13)


def test_linear_profile_plus_mode():
    N = 32
    H = 2 * math.pi / N
    K = np.tile([0.3, 0.0, 0.6], (N * N, 1))
    i, j = np.arange(N), np.arange(N)
    lin = np.tile(2.0 - 3.0 * i / N, (N, 1))            # u_left = 2, u_right = -1
    mode = np.sin(math.pi * 4 * i / N)[None, :] * np.sin(2 * H * j)[:, None]
    dt, s = 0.02, 80
    U = oracle.macro_run_dirichlet(lin + mode, K, dt, s, 2.0, -1.0)
    z = -dt * (4 * 0.3 * math.sin(math.pi * 4 / (2 * N)) ** 2
               + 4 * 0.6 * math.sin(H) ** 2) / H ** 2
    np.testing.assert_allclose(U, lin + mode * (1 + z + z * z / 2) ** s, atol=1e-13)


def test_x1_dependent_K_reduces_to_1d():
    # K varies along x1 only (with a cross term); U depends on x1 only, so the
    # 2-D flux form is the 1-D scheme d/dt U_i = (F_{i+1/2} - F_{i-1/2}) / H,
    # F_{i+1/2} = (K11_i + K11_{i+1})/2 (U_{i+1} - U_i) / H, U_0 = 1, U_N = 0
    N = 32
    H = 2 * math.pi / N
    x = H * np.arange(N)
    k11 = 0.5 + 0.3 * np.sin(x) + 0.1 * np.cos(3 * x)
    k12 = 0.2 * np.cos(2 * x)
    k22 = 0.8 + 0.2 * np.sin(x)
    K = np.stack([np.tile(k11, N), np.tile(k12, N), np.tile(k22, N)], 1)
    U0 = flows.step_u0(N)
    dt, s = 0.2 * H * H / 1.0, 300
    U = oracle.macro_run_dirichlet(U0, K, dt, s, 1.0, 0.0)
    kf = 0.5 * (k11 + np.roll(k11, -1))                  # face i+1/2 (periodic K field)

    def rhs(u):
        ue = np.append(u, 0.0)                          # u_N = u_right
        F = kf * (ue[1:] - ue[:-1]) / H                 # F_{i+1/2}, i = 0..N-1
        r = np.zeros(N)
        r[1:] = (F[1:] - F[:-1]) / H
        return r
    u1 = _heun_1d(U0[0].copy(), rhs, dt, s)
    np.testing.assert_allclose(U, np.tile(u1, (N, 1)), atol=1e-13)
    assert 0.05 < u1[N // 2 + 2] < 0.95                  # the step has spread


def test_dns_without_flow_equals_macro_with_kappa():
    N, kappa = 32, 0.4
    U0 = flows.step_u0(N)
    rng = np.random.default_rng(3)
    U0 = U0 + 0.1 * rng.standard_normal((N, N))
    dt, s = 0.01, 70
    u = oracle.dns_run_dirichlet(np.zeros((N, N)), kappa, dt, s, U0, 1.0, 0.0)
    U = oracle.macro_run_dirichlet(U0, np.tile([kappa, 0.0, kappa], (N * N, 1)), dt, s, 1.0, 0.0)
    np.testing.assert_allclose(u, U, atol=1e-14)


def test_dns_shear_rows_are_1d_central_advection():
    # psi = A sin(m x2): v = (v1(x2), 0) with v1 = -A cos(m x2) sin(m h)/h; with
    # kappa = 0 each row j is u_t = c_j D0x u with u_0 = 1 and u_N = 0
    N, A, m = 32, 0.6, 2
    h = 2 * math.pi / N
    psi = oracle.grid_psi(flows.shear_x2(A, m), N)
    x = h * np.arange(N)
    c = -A * np.cos(m * x) * math.sin(m * h) / h
    U0 = flows.step_u0(N)
    dt, s = 0.02, 120
    u = oracle.dns_run_dirichlet(psi, 0.0, dt, s, U0, 1.0, 0.0)
    for j in range(N):
        def rhs(r, cj=c[j]):
            e = np.concatenate([r, [0.0]])
            out = np.zeros(N)
            out[1:] = cj * (e[2:] - e[:-2]) / (2 * h)
            return out
        np.testing.assert_allclose(u[j], _heun_1d(U0[j].copy(), rhs, dt, s), atol=1e-13)
    assert np.abs(u - U0).max() > 0.1


def test_dns_shear_across_x1_only_diffuses_a_step():
    # psi = A sin(m x1): v = (0, v2(x1)) does not move an x2-independent field;
    # the step then diffuses as with v = 0
    N, kappa = 32, 0.3
    psi = oracle.grid_psi(flows.shear_x1(0.8, 3), N)
    U0 = flows.step_u0(N)
    u = oracle.dns_run_dirichlet(psi, kappa, 0.01, 90, U0, 1.0, 0.0)
    w = oracle.dns_run_dirichlet(np.zeros((N, N)), kappa, 0.01, 90, U0, 1.0, 0.0)
    np.testing.assert_allclose(u, w, atol=1e-14)
