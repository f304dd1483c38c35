"""GPU parity of the solvers with the Sec. 4 boundary conditions (Dirichlet in
x1, periodic in x2) against the oracle: the macro step on the resident
(N <= 64) and the per-stage (N > 64) paths in both precisions, and the direct
simulation, from the step initial condition."""
import numpy as np
import pytest

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


@pytest.mark.parametrize("N,prec,tol", [(32, "fp64", 1e-12), (48, "fp32", 1e-5),
                                        (96, "fp64", 1e-12), (128, "fp32", 1e-5)])
def test_macro_dirichlet_parity(mlsd, torch_mod, N, prec, tol):
    dev = torch_mod.device("cuda:0")
    dtype = torch_mod.float64 if prec == "fp64" else torch_mod.float32
    K = random_spd(N * N, np.random.default_rng(N + 7), 0.1, 1.0)
    U0 = flows.step_u0(N)
    U0[:, 0] = 0.3                                   # overwritten by the boundary value
    dt = oracle.macro_dt(K, N, 0.2)
    ns = 80
    Ug = torch_mod.tensor(U0, dtype=dtype, device=dev)
    Kg = torch_mod.tensor(K, dtype=torch_mod.float64, device=dev)
    mlsd.macro_step_dirichlet(Ug, Kg, dt, ns, 1.0, 0.0)
    Ur = oracle.macro_run_dirichlet(U0, K, dt, ns, 1.0, 0.0)
    got = Ug.cpu().numpy()
    assert np.all(got[:, 0] == 1.0)
    assert rel_l2(got, Ur) < tol


def test_macro_dirichlet_linear_profile_steady(mlsd, torch_mod):
    N = 80
    K = np.tile([0.6, 0.25, 0.4], (N * N, 1))
    U0 = np.tile(1.0 - np.arange(N) / N, (N, 1))
    Ug = torch_mod.tensor(U0, dtype=torch_mod.float64, device="cuda:0")
    Kg = torch_mod.tensor(K, dtype=torch_mod.float64, device="cuda:0")
    mlsd.macro_step_dirichlet(Ug, Kg, 0.001, 50, 1.0, 0.0)
    assert np.abs(Ug.cpu().numpy() - U0).max() < 1e-13


@pytest.mark.parametrize("nf,steps,prec,tol", [(128, 200, "fp32", 1e-5), (200, 60, "fp32", 1e-5),
                                               (128, 300, "fp64", 1e-12)])
def test_dns_dirichlet_parity(mlsd, torch_mod, nf, steps, prec, tol):
    dev = torch_mod.device("cuda:0")
    spec = flows.cellular_two_scale(1.0 / 3, 1.0 / 3, 5)
    kappa = 1.0
    psi = oracle.grid_psi(spec, nf)
    h = 2 * np.pi / nf
    dt = 0.2 * min(h * h / (4 * kappa), h / 2.0)
    U0 = flows.step_u0(nf)
    dtype = torch_mod.float64 if prec == "fp64" else torch_mod.float32
    u = torch_mod.tensor(U0, dtype=dtype, device=dev)
    ut = torch_mod.empty_like(u)
    pg = torch_mod.tensor(psi, dtype=torch_mod.float32, device=dev)
    mlsd.dns_run_dirichlet(u, ut, pg, kappa, dt, steps, 1.0, 0.0)
    torch_mod.cuda.synchronize()
    # the oracle on the FP32-rounded stream function the kernel reads
    psi32 = pg.double().cpu().numpy()
    ref = oracle.dns_run_dirichlet(psi32 if prec == "fp64" else psi, kappa, dt, steps, U0, 1.0, 0.0)
    got = u.cpu().numpy()
    assert np.all(got[:, 0] == 1.0)
    assert rel_l2(got, ref) < tol
    assert np.abs(ref - U0).max() > 0.1


def test_dirichlet_argument_checks(mlsd, torch_mod):
    lib = mlsd.lib()
    u = torch_mod.zeros(8, 8, dtype=torch_mod.float32, device="cuda:0")
    K = torch_mod.zeros(64, 3, dtype=torch_mod.float64, device="cuda:0")
    s = torch_mod.cuda.current_stream().cuda_stream
    assert lib.mlsd_macro_step_dirichlet(8, u.data_ptr(), 0, K.data_ptr(), -1.0, 1, 1.0, 0.0,
                                         None, s) == -1
    assert lib.mlsd_macro_step_dirichlet(8, u.data_ptr(), 0, K.data_ptr(), 0.1, 1,
                                         float("nan"), 0.0, None, s) == -1
    # u and its scratch buffer alias
    assert lib.mlsd_dns_run_dirichlet(8, u.data_ptr(), u.data_ptr(), u.data_ptr(), 0, 1.0, 0.1,
                                      1, 1.0, 0.0, s) == -1
    # a precision other than FP32 / FP64
    t = torch_mod.zeros_like(u)
    assert lib.mlsd_dns_run_dirichlet(8, u.data_ptr(), t.data_ptr(), u.data_ptr(), 2, 1.0, 1e-4,
                                      1, 1.0, 0.0, s) == -1
