"""The oracle's pins applied to the GPU's own output: discrete shear closed
forms with a full-tensor base, the symmetry of the cellular flow, positive
semidefinite enhancement K - B, conservation of the corrector's mean, and the
energy form of the correctors (equal to K - B for a shear)."""
import math

import numpy as np
import pytest

import inputs
from inputs import flows
import oracle
from tests._parity import random_spd

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch_mod():
    import torch
    assert torch.cuda.is_available()
    return torch


@pytest.fixture(scope="module")
def mlsd():
    import paper_1510_00451_gb300 as m
    return m


def _transient(z, nb, na):
    # Heun's amplification g = 1 - z + z^2/2 of a decaying mode, averaged over the window
    g = 1 - z + z * z / 2
    return g ** (nb + 1) * (1 - g ** na) / ((1 - g) * na)


def _solve(torch, lv, level, B, w_dtype=None):
    dev = torch.device("cuda:0")
    Kb = torch.tensor(B, dtype=torch.float64, device=dev)
    Ko = torch.zeros_like(Kb)
    n = lv.info(level)["n"]
    w = torch.zeros(lv.P, 2, n, n, dtype=w_dtype, device=dev) if w_dtype is not None else None
    lv.solve_level(level, Kb, Ko, w)
    assert lv.status() == 0
    return Ko.cpu().numpy(), (None if w is None else w.cpu().numpy())


@pytest.mark.parametrize("axis", [1, 2])
@pytest.mark.parametrize("prec,tol", [("fp32", 2e-6), ("fp64", 1e-12)])
def test_shear_closed_forms_on_gpu(mlsd, torch_mod, axis, prec, tol):
    # psi = A sin(m x_axis): K_jj = B_jj + A^2 cos^2(m h/2) / (2 B_ii) (1 - transient),
    # i the shear direction, j the other; the rest of K equals B
    A, m, N, n, nb, na = 0.6, 3, 2, 32, 300, 200
    spec = flows.shear_x1(A, m) if axis == 1 else flows.shear_x2(A, m)
    lv = mlsd.Levels(spec, 0.1, N, [1, 8], [n], n_burn_fixed=nb, n_avg_fixed=na, precision=prec)
    B0 = np.array([0.3, 0.07, 0.2])
    K, _ = _solve(torch_mod, lv, 1, np.tile(B0, (N * N, 1)))
    h = 2 * math.pi / n
    Bii = B0[0] if axis == 1 else B0[2]
    sig = A * math.sin(m * h) / h                       # amplitude of the discrete velocity
    dt = oracle.micro_dt(h, sig, B0, 0.2)
    lam = 4 * Bii * math.sin(m * h / 2) ** 2 / h ** 2
    enh = A ** 2 * math.cos(m * h / 2) ** 2 / (2 * Bii) * (1 - _transient(dt * lam, nb, na))
    want = B0 + (np.array([0, 0, enh]) if axis == 1 else np.array([enh, 0, 0]))
    for p in range(N * N):
        np.testing.assert_allclose(K[p], want, rtol=tol, atol=tol * want.max())


def test_cellular_symmetry_on_gpu(mlsd, torch_mod):
    # sin x sin y is symmetric under x1 <-> x2 and odd under x1 -> -x1: with B = kappa I,
    # K11 = K22 and K12 = 0 up to FP32 rounding, and K exceeds B
    N, n = 2, 64
    lv = mlsd.Levels(flows.cellular_two_scale(1.0, 0.0, 1), 0.05, N, [1, 4], [n],
                     n_burn_fixed=2000, n_avg_fixed=1000)
    K, _ = _solve(torch_mod, lv, 1, np.tile([0.05, 0.0, 0.05], (N * N, 1)))
    for p in range(N * N):
        assert abs(K[p, 0] - K[p, 2]) < 2e-6 * K[p, 0]
        assert abs(K[p, 1]) < 2e-6 * K[p, 0]
        assert K[p, 0] > 0.05


def test_enhancement_is_positive_semidefinite_on_gpu(mlsd, torch_mod):
    # continuous spectrum, random full-tensor bases, the full relaxation window:
    # sym(<v w>) = K - B is positive semidefinite (up to the e^-8 transient left)
    spec = flows.continuous_spectrum(40, seed=3)
    N = 6
    lv = mlsd.Levels(spec, 2e-3, N, [1, 4, 16, 41], [32, 32, 32])
    B = inputs.random_bases(N * N, 2e-3, 11)
    for level in (2, 3):
        K, _ = _solve(torch_mod, lv, level, B)
        for p in range(N * N):
            D = np.array([[K[p, 0] - B[p, 0], K[p, 1] - B[p, 1]], [K[p, 1] - B[p, 1], K[p, 2] - B[p, 2]]])
            assert np.linalg.eigvalsh(D).min() > -1e-4 * (B[p, 0] + B[p, 2]), (level, p, D)


def test_corrector_mean_is_conserved_on_gpu(mlsd, torch_mod):
    # the discrete velocity is divergence free and the source has zero mean, so
    # sum_ab w_j stays at zero (FP32 rounding only)
    spec = flows.cellular_two_scale(1.0, 0.5, 3)
    N = 3
    lv = mlsd.Levels(spec, 0.05, N, [1, 8], [32], n_burn_fixed=300, n_avg_fixed=100)
    B = random_spd(N * N, np.random.default_rng(2), 0.03, 0.1)
    _, w = _solve(torch_mod, lv, 1, B, torch_mod.float32)
    for p in range(N * N):
        for j in range(2):
            assert abs(w[p, j].sum(dtype=np.float64)) < 1e-5 * np.abs(w[p, j]).sum(dtype=np.float64)
        assert np.abs(w[p]).max() > 1e-3


@pytest.mark.parametrize("prec,tol", [("fp32", 2e-5), ("fp64", 1e-10)])
def test_energy_form_on_gpu(mlsd, torch_mod, prec, tol):
    # the energy form of the GPU's own correctors: for a diagonal shear with a
    # full-tensor base it equals K - B (the correctors are not advected), and
    # for a general flow it matches the oracle's energy form of the oracle's
    # correctors on the same patches
    dev = torch_mod.device("cuda:0")
    dtype = torch_mod.float64 if prec == "fp64" else torch_mod.float32
    N, n = 2, 32
    lv = mlsd.Levels(flows.shear_diag(0.6, 2), 0.1, N, [1, 8], [n], n_burn_fixed=3000,
                     n_avg_fixed=500, precision=prec)
    B = np.tile([0.3, 0.08, 0.2], (N * N, 1))
    Bd = torch_mod.tensor(B, dtype=torch_mod.float64, device=dev)
    K = torch_mod.zeros_like(Bd)
    w = torch_mod.zeros(N * N, 2, n, n, dtype=dtype, device=dev)
    lv.solve_level(1, Bd, K, w)
    E = torch_mod.zeros_like(Bd)
    M = torch_mod.zeros(N * N, 2, dtype=torch_mod.float64, device=dev)
    lv.corrector_energy(1, Bd, w, E, M)
    assert lv.status() == 0
    Kc, Ec = K.cpu().numpy(), E.cpu().numpy()
    for p in range(N * N):
        np.testing.assert_allclose(Ec[p], Kc[p] - B[p], rtol=tol, atol=tol * np.abs(Kc[p] - B[p]).max())
    mtol = 2e-5 if prec == "fp32" else 1e-12
    assert np.abs(M.cpu().numpy()).max() < mtol * float(w.abs().max())

    spec = flows.cellular_two_scale(0.8, 0.5, 4)
    edges, pn, N = [1, 4, 8], [n, n], 3
    lv = mlsd.Levels(spec, 0.03, N, edges, pn, n_burn_fixed=200, n_avg_fixed=100, precision=prec)
    B = random_spd(N * N, np.random.default_rng(4), 0.03, 0.1)
    Bd = torch_mod.tensor(B, dtype=torch_mod.float64, device=dev)
    K = torch_mod.zeros_like(Bd)
    w = torch_mod.zeros(N * N, 2, n, n, dtype=dtype, device=dev)
    lv.solve_level(2, Bd, K, w)
    E = torch_mod.zeros_like(Bd)
    lv.corrector_energy(2, Bd, w, E)
    Ec = E.cpu().numpy()
    from tests._parity import oracle_level, level_geometry, rel_l2
    ref = oracle_level(spec, edges, pn, 2, N, B, list(range(N * N)), n_burn_fixed=200,
                       n_avg_fixed=100, want_w=True)
    h = level_geometry(edges, pn, 2)[2]
    for p, (_, w_or) in enumerate(ref):
        E_or, _ = oracle.corrector_energy(w_or, h, B[p])
        assert rel_l2(Ec[p], E_or) < (1e-4 if prec == "fp32" else 1e-10), (p, Ec[p], E_or)
