"""GPU parity of the macro solver (Eq. homo), the direct simulation (Eq. model),
the grid synthesis of psi and the coarse-graining, against the oracle."""
import math

import numpy as np
import pytest

import inputs
from inputs import flows
import oracle
from tests._parity import rel_l2, random_spd

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


def _K_field(N, seed):
    return random_spd(N * N, np.random.default_rng(seed), 0.1, 1.0)


@pytest.mark.parametrize("N,prec,tol", [(32, "fp64", 1e-12), (64, "fp32", 1e-5),
                                        (128, "fp32", 1e-5), (128, "fp64", 1e-12),
                                        (20, "fp64", 1e-12)])
def test_macro_parity(mlsd, torch_mod, N, prec, tol):
    dev = torch_mod.device("cuda:0")
    dtype = torch_mod.float64 if prec == "fp64" else torch_mod.float32
    K = _K_field(N, N)
    U0 = flows.gaussian_u0(N)
    dt = oracle.macro_dt(K, N, 0.2)
    ns = 60
    Ug = torch_mod.tensor(U0, dtype=dtype, device=dev)
    Kg = torch_mod.tensor(K, dtype=torch_mod.float64, device=dev)
    mass = mlsd.macro_step(Ug, Kg, dt, ns)
    Ur, mr = oracle.macro_run(U0, K, dt, ns)
    assert rel_l2(Ug.cpu().numpy(), Ur) < tol
    # conservation of H^2 sum(U) in the FP64 mass record
    mtol = 1e-13 if prec == "fp64" else 1e-6
    assert np.max(np.abs(mass - mass[0])) < mtol * mass[0]
    np.testing.assert_allclose(mass[0], mr[0], rtol=1e-7 if prec == "fp32" else 1e-14)


def test_macro_dt_matches_rule(mlsd, torch_mod):
    N = 48
    K = _K_field(N, 3)
    Kg = torch_mod.tensor(K, dtype=torch_mod.float64, device="cuda:0")
    assert mlsd.macro_dt(Kg, N, 0.2) == pytest.approx(oracle.macro_dt(K, N, 0.2), rel=1e-15)


def test_macro_zero_steps_and_no_mass(mlsd, torch_mod):
    N = 128
    U0 = flows.gaussian_u0(N)
    Ug = torch_mod.tensor(U0, dtype=torch_mod.float32, device="cuda:0")
    Kg = torch_mod.tensor(_K_field(N, 1), dtype=torch_mod.float64, device="cuda:0")
    m = mlsd.macro_step(Ug, Kg, 0.01, 0)
    assert len(m) == 1 and np.array_equal(Ug.cpu().numpy(), U0.astype(np.float32))
    assert mlsd.macro_step(Ug, Kg, 0.001, 3, want_mass=False) is None


def test_grid_psi_parity(mlsd, torch_mod):
    spec = flows.continuous_spectrum(48, seed=2)
    nf = 256
    g = torch_mod.zeros(nf, nf, dtype=torch_mod.float32, device="cuda:0")
    mlsd.grid_psi(spec, nf, g)
    ref = oracle.grid_psi(spec, nf)
    assert np.abs(g.cpu().numpy() - ref).max() < 1e-6 * np.abs(ref).max()


@pytest.mark.parametrize("nf,steps", [(512, 120), (128, 300)])
def test_dns_parity(mlsd, torch_mod, nf, steps):
    # the Sec. 4 reference grid size; FP32 on the GPU against the FP64 oracle
    spec = flows.cellular_two_scale(1.0, 0.3, 8)
    kappa = 0.02
    psi_r = oracle.grid_psi(spec, nf)
    h = 2 * math.pi / nf
    v1, v2 = oracle.velocity(psi_r, h)
    dt = 0.2 * min(h / np.max(np.abs(v1) + np.abs(v2)), h * h / (4 * kappa))
    u0 = flows.gaussian_u0(nf)
    ur = oracle.dns_run(psi_r, kappa, dt, steps, u0)
    dev = torch_mod.device("cuda:0")
    psi = torch_mod.zeros(nf, nf, dtype=torch_mod.float32, device=dev)
    mlsd.grid_psi(spec, nf, psi)
    assert mlsd.dns_dt(psi, kappa, 0.2) == pytest.approx(dt, rel=1e-6)
    u = torch_mod.tensor(u0, dtype=torch_mod.float32, device=dev)
    ut = torch_mod.empty_like(u)
    mlsd.dns_run(u, ut, psi, kappa, dt, steps)
    assert mlsd.dns_status() == 0
    assert rel_l2(u.cpu().numpy(), ur) < 1e-5
    # coarse-graining and the FP64 mass
    N = 32
    Ug = torch_mod.zeros(N, N, dtype=torch_mod.float32, device=dev)
    m = mlsd.coarse_grain(u, N, Ug)
    Ucr, mr = oracle.coarse_grain(ur, N)
    assert rel_l2(Ug.cpu().numpy(), Ucr) < 1e-5
    assert m == pytest.approx(mr, rel=1e-6)
    m0 = oracle.coarse_grain(u0, N)[1]
    assert m == pytest.approx(m0, rel=1e-5)       # the DNS conserves sum(u)


_DNS_REF = {}


@pytest.mark.parametrize("kind", ["64", "32", "t32", "t32x2", "t64", "t32p"])
@pytest.mark.parametrize("nf,steps", [(256, 40), (2048, 6)])
def test_dns_kernels_parity(mlsd, torch_mod, monkeypatch, kind, nf, steps):
    # every DNS kernel, forced one at a time: per-tile CTAs staged by cp.async (64- and
    # 32-row tiles) and persistent CTAs fed by tensor copies (one or two staging buffers).
    # At 256^2 every tile touches the grid's edge (periodic images filled in after the
    # copy); at 2048^2 most tiles are interior and each persistent CTA walks several
    monkeypatch.setenv("MLSD_DNS_TY", kind)
    spec = flows.cellular_two_scale(1.0, 0.3, 8)
    kappa = 0.02
    h = 2 * math.pi / nf
    if nf not in _DNS_REF:
        psi_r = oracle.grid_psi(spec, nf)
        v1, v2 = oracle.velocity(psi_r, h)
        dt = 0.2 * min(h / np.max(np.abs(v1) + np.abs(v2)), h * h / (4 * kappa))
        u0 = flows.gaussian_u0(nf)
        _DNS_REF[nf] = (dt, u0, oracle.dns_run(psi_r, kappa, dt, steps, u0))
    dt, u0, ur = _DNS_REF[nf]
    dev = torch_mod.device("cuda:0")
    psi = torch_mod.zeros(nf, nf, dtype=torch_mod.float32, device=dev)
    mlsd.grid_psi(spec, nf, psi)
    u = torch_mod.tensor(u0, dtype=torch_mod.float32, device=dev)
    ut = torch_mod.empty_like(u)
    mlsd.dns_run(u, ut, psi, kappa, dt, steps)
    assert mlsd.dns_status() == 0
    assert rel_l2(u.cpu().numpy(), ur) < 1e-5


@pytest.mark.slow
def test_two_scale_cellular_fp64_end_to_end(mlsd, torch_mod):
    # 32 x 32 macro grid, 2 levels of 32^2 patches (1024 per level), FP64, full window,
    # then the macro solve to T = 1 from the Gaussian initial condition
    cfg = inputs.config_problem("two_scale_cellular_fp64")
    N = cfg["n_macro"]
    dev = torch_mod.device("cuda:0")
    lv = mlsd.Levels(cfg["spectrum"], cfg["kappa"], N, cfg["edges"], cfg["patch_n"],
                     cfl=cfg["cfl"], precision="fp64")
    K = torch_mod.zeros(N * N, 3, dtype=torch_mod.float64, device=dev)
    lv.effective_diffusivity(K)
    assert lv.status() == 0
    Kg = K.cpu().numpy()
    nodes = [(0, 0), (9, 30), (31, 17)]
    Kr = oracle.chain(cfg["spectrum"], cfg["edges"], cfg["patch_n"], N, cfg["kappa"], nodes,
                      cfl=cfg["cfl"])
    for (i, j), kr in zip(nodes, Kr):
        assert rel_l2(Kg[j * N + i], kr) < 1e-10
    # translation invariance: one K everywhere (the oracle pin P10)
    assert np.abs(Kg - Kg[0]).max() < 1e-10 * np.abs(Kg[0]).max()
    # macro step with the oracle's K on every node
    Ko = np.tile(Kr[0], (N * N, 1))
    dt = oracle.macro_dt(Ko, N, cfg["cfl"])
    ns = math.ceil(cfg["T"] / dt)
    U0 = flows.gaussian_u0(N, cfg["sigma"])
    Ur, mr = oracle.macro_run(U0, Ko, cfg["T"] / ns, ns)
    Ug = torch_mod.tensor(U0, dtype=torch_mod.float64, device=dev)
    mg = mlsd.macro_step(Ug, K, cfg["T"] / ns, ns)
    assert rel_l2(Ug.cpu().numpy(), Ur) < 1e-9
    assert np.max(np.abs(mg - mg[0])) < 1e-13 * mg[0]


@pytest.mark.slow
def test_dns_full_grid_conserves_mass(mlsd, torch_mod):
    # the 8192^2 grid of the DNS workload (the oracle cannot follow it step by step
    # at this size): 50 fused steps keep sum(u) to FP32 rounding and stay finite,
    # and the coarse-grained field stays close to the one of the first step's start
    cfg = inputs.config_problem("continuous_spectrum")
    nf, kappa = 8192, cfg["kappa"]
    dev = torch_mod.device("cuda:0")
    psi = torch_mod.empty(nf, nf, dtype=torch_mod.float32, device=dev)
    mlsd.grid_psi(cfg["spectrum"], nf, psi)
    dt = mlsd.dns_dt(psi, kappa, cfg["cfl"])
    u = torch_mod.tensor(flows.gaussian_u0(nf, cfg["sigma"]), dtype=torch_mod.float32, device=dev)
    ut = torch_mod.empty_like(u)
    N = cfg["n_macro"]
    U0 = torch_mod.zeros(N, N, dtype=torch_mod.float32, device=dev)
    m0 = mlsd.coarse_grain(u, N, U0)
    mlsd.dns_run(u, ut, psi, kappa, dt, 50)
    U = torch_mod.zeros_like(U0)
    m = mlsd.coarse_grain(u, N, U)
    assert bool(torch_mod.isfinite(u).all())
    assert m == pytest.approx(m0, rel=1e-6)
    assert rel_l2(U.cpu().numpy(), U0.cpu().numpy()) < 1e-2      # 50 steps of dt ~ 3e-5
