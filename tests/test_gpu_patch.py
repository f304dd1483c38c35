"""GPU parity of the batched patch solves and the level chain against the oracle.

Tolerances (those the library states for its results): relative L2 <= 1e-5 on the corrector
fields w, relative <= 1e-4 on K_eff, for the FP32 stencil with FP64 averages;
the FP64 path is held to 1e-10.
"""
import math

import numpy as np
import pytest

import inputs
from inputs import flows
import oracle
from tests._parity import oracle_level, random_spd, rel_l2, level_geometry

pytestmark = pytest.mark.gpu

W_TOL, K_TOL, FP64_TOL = 1e-5, 1e-4, 1e-10


@pytest.fixture(scope="module")
def torch_mod():
    import torch
    assert torch.cuda.is_available()
    return torch


@pytest.fixture(scope="module")
def mlsd():
    import paper_1510_00451_gb300 as m
    return m


def _solve(mlsd, torch, lv, level, B, want_w, dtype):
    dev = torch.device("cuda:0")
    Kb = torch.tensor(B, dtype=torch.float64, device=dev)
    Ko = torch.zeros_like(Kb)
    n = lv.info(level)["n"]
    w = torch.zeros(lv.P, 2, n, n, dtype=dtype, device=dev) if want_w else None
    lv.solve_level(level, Kb, Ko, w)
    assert lv.status() == 0
    torch.cuda.synchronize()
    return Ko.cpu().numpy(), (None if w is None else w.cpu().numpy())


@pytest.mark.parametrize("level", [1, 2, 3])
def test_level_parity_fp32_n64(mlsd, torch_mod, level):
    # 3-level cellular hierarchy, 5 x 5 macro grid (odd: snapping ties), random SPD bases
    spec = flows.cellular_hierarchy(3, 4)
    edges, pn, N = [1, 4, 16, 64], [64, 64, 64], 5
    lv = mlsd.Levels(spec, 0.01, N, edges, pn, n_burn_fixed=150, n_avg_fixed=120)
    B = random_spd(N * N, np.random.default_rng(level))
    K, w = _solve(mlsd, torch_mod, lv, level, B, True, torch_mod.float32)
    patches = [0, 7, 13, 24]
    ref = oracle_level(spec, edges, pn, level, N, B, patches, n_burn_fixed=150, n_avg_fixed=120,
                       want_w=True)
    for p, (Kr, wr) in zip(patches, ref):
        assert rel_l2(K[p], Kr) < K_TOL, (p, K[p], Kr)
        assert rel_l2(w[p, 0], wr[0]) < W_TOL and rel_l2(w[p, 1], wr[1]) < W_TOL


def test_level_parity_fp32_n32_continuous_spectrum(mlsd, torch_mod):
    # octave bands of a random-phase spectrum: not periodic on the patch (seam wraps)
    spec = flows.continuous_spectrum(24, seed=11)
    edges, pn, N = [1, 2, 4, 8, 16, 25], [32] * 5, 3
    lv = mlsd.Levels(spec, 2e-3, N, edges, pn, n_burn_fixed=100, n_avg_fixed=100)
    for level in (1, 3, 5):
        B = random_spd(N * N, np.random.default_rng(10 + level), 0.002, 0.006)
        K, w = _solve(mlsd, torch_mod, lv, level, B, True, torch_mod.float32)
        patches = list(range(N * N))
        ref = oracle_level(spec, edges, pn, level, N, B, patches, n_burn_fixed=100,
                           n_avg_fixed=100, want_w=True)
        for p, (Kr, wr) in zip(patches, ref):
            assert rel_l2(K[p], Kr) < K_TOL, (level, p, K[p], Kr)
            assert rel_l2(w[p], wr) < W_TOL, (level, p)


@pytest.mark.parametrize("n", [32, 64])
def test_level_parity_fp64(mlsd, torch_mod, n):
    spec = flows.cellular_two_scale(1.0, 1.0, 8)
    edges, pn, N = [1, 8, 9], [n, n], 4
    lv = mlsd.Levels(spec, 0.05, N, edges, pn, n_burn_fixed=200, n_avg_fixed=100,
                     precision="fp64")
    for level in (1, 2):
        B = random_spd(N * N, np.random.default_rng(n + level), 0.05, 0.2)
        K, w = _solve(mlsd, torch_mod, lv, level, B, True, torch_mod.float64)
        patches = [0, 5, 15]
        ref = oracle_level(spec, edges, pn, level, N, B, patches, n_burn_fixed=200,
                           n_avg_fixed=100, want_w=True)
        for p, (Kr, wr) in zip(patches, ref):
            assert rel_l2(K[p], Kr) < FP64_TOL
            assert rel_l2(w[p], wr) < FP64_TOL


def test_kappa_only_limit_exact(mlsd, torch_mod):
    # no modes: v = 0, w stays 0 and K equals the base bit for bit
    spec = flows.Spectrum(np.zeros(0, np.int32), np.zeros(0, np.int32), np.zeros(0), np.zeros(0))
    lv = mlsd.Levels(spec, 0.02, 4, [1, 4], [64], n_burn_fixed=10, n_avg_fixed=10)
    B = random_spd(16, np.random.default_rng(0))
    K, w = _solve(mlsd, torch_mod, lv, 1, B, True, torch_mod.float32)
    assert np.array_equal(K, B)
    assert not np.any(w)


@pytest.mark.parametrize("prec,tol", [("fp32", 2e-6), ("fp64", 1e-12)])
def test_diagonal_shear_closed_form_on_gpu(mlsd, torch_mod, prec, tol):
    # psi = A sin(m (x1 + x2)) as the level's diagonal band: K is known in closed form
    A, m, N, n = 0.8, 3, 3, 32
    spec = flows.shear_diag(A, m)
    lv = mlsd.Levels(spec, 0.1, N, [1, 8], [n], n_burn_fixed=400, n_avg_fixed=300, precision=prec)
    B = np.tile([0.3, 0.08, 0.2], (N * N, 1))
    K, _ = _solve(mlsd, torch_mod, lv, 1, B, False, torch_mod.float32)
    h = 2 * math.pi / n
    mu = (4 * (B[0, 0] + B[0, 2]) * math.sin(m * h / 2) ** 2 + 2 * B[0, 1] * math.sin(m * h) ** 2) / h ** 2
    sig = A * math.sin(m * h) / h
    dt = oracle.micro_dt(h, 2 * sig, B[0], 0.2)
    z = dt * mu
    g = 1 - z + z * z / 2
    T = g ** 401 * (1 - g ** 300) / ((1 - g) * 300)
    e = sig ** 2 / (2 * mu) * (1 - T)
    want = np.array([B[0, 0] + e, B[0, 1] - e, B[0, 2] + e])
    for p in range(N * N):
        assert rel_l2(K[p], want) < tol, (K[p], want)


def test_bad_base_latches_error(mlsd, torch_mod):
    # an indefinite base gives no time step: the kernel latches MLSD_EINVAL and
    # returns without stepping; the context stays usable
    spec = flows.cellular_two_scale(1.0, 0.0, 1)
    lv = mlsd.Levels(spec, 0.05, 2, [1, 4], [32])
    dev = torch_mod.device("cuda:0")
    Kb = torch_mod.tensor([[0.1, 0.0, 0.1]] * 3 + [[0.1, 0.5, 0.1]], dtype=torch_mod.float64, device=dev)
    Ko = torch_mod.zeros_like(Kb)
    lv.solve_level(1, Kb, Ko)
    assert lv.status() == -1
    assert lv.status() == 0          # cleared after reading
    Kb[3] = torch_mod.tensor([0.1, 0.0, 0.1], dtype=torch_mod.float64)
    lv2 = mlsd.Levels(spec, 0.05, 2, [1, 4], [32], n_burn_fixed=5, n_avg_fixed=5)
    lv2.solve_level(1, Kb, Ko)
    assert lv2.status() == 0


def _chain_check(mlsd, torch, spec, edges, pn, N, kappa, nodes, tol, prec="fp32", **kw):
    lv = mlsd.Levels(spec, kappa, N, edges, pn, precision=prec, **kw)
    dev = torch.device("cuda:0")
    K = torch.zeros(N * N, 3, dtype=torch.float64, device=dev)
    Kl = torch.zeros(len(edges) - 1, N * N, 3, dtype=torch.float64, device=dev)
    lv.effective_diffusivity(K, Kl)
    assert lv.status() == 0
    K = K.cpu().numpy()
    okw = {}
    if kw.get("n_avg_fixed", 0) > 0:
        okw = dict(n_burn_fixed=kw["n_burn_fixed"], n_avg_fixed=kw["n_avg_fixed"])
    if kw.get("patch_div") is not None:
        okw["patch_div"] = kw["patch_div"]
    if kw.get("periodize"):
        okw["periodize"] = True
    want = oracle.chain(spec, edges, pn, N, kappa, nodes, **okw)
    for (i, j), wv in zip(nodes, want):
        assert rel_l2(K[j * N + i], wv) < tol, ((i, j), K[j * N + i], wv)
    return K, Kl.cpu().numpy()


def test_chain_parity_two_scale_fp64(mlsd, torch_mod):
    _chain_check(mlsd, torch_mod, flows.cellular_two_scale(1.0, 1.0, 8), [1, 8, 9], [32, 32], 4,
                 0.05, [(0, 0), (1, 3), (3, 2)], FP64_TOL, prec="fp64",
                 n_burn_fixed=300, n_avg_fixed=200)


def test_chain_parity_three_level_fp32(mlsd, torch_mod):
    _chain_check(mlsd, torch_mod, flows.cellular_hierarchy(3, 4), [1, 4, 16, 64], [64] * 3, 3,
                 0.01, [(0, 0), (2, 1)], K_TOL, n_burn_fixed=300, n_avg_fixed=200)


def test_chain_with_off_diagonal_parts(mlsd, torch_mod):
    # Algorithms 1-3 with a psi_12 part at level 1 (the oracle pin's closed-form flow)
    spec = flows.combine(flows.shear_diag(0.6, 1), flows.shear_diag(0.35, 4), flows.shear_x2(0.3, 8))
    _chain_check(mlsd, torch_mod, spec, [1, 4, 16], [32, 32], 4, 0.05,
                 [(0, 0), (1, 2), (3, 1)], K_TOL, n_burn_fixed=300, n_avg_fixed=200)


def test_chain_continuous_spectrum_with_offdiagonals(mlsd, torch_mod):
    spec = flows.continuous_spectrum(24, seed=5)
    _chain_check(mlsd, torch_mod, spec, [1, 2, 4, 8, 16, 25], [32] * 5, 3, 2e-3,
                 [(0, 0), (1, 2), (2, 2)], K_TOL, n_burn_fixed=120, n_avg_fixed=80)


@pytest.mark.slow
def test_full_three_level_cellular_sampled(mlsd, torch_mod):
    # 128 x 128 macro grid, 64^2 patches, 16384 patches per level, full tau window
    # (the benchmark's launch configuration); sampled nodes against the oracle
    cfg = inputs.config_problem("three_level_cellular")
    N = cfg["n_macro"]
    K, Kl = _chain_check(mlsd, torch_mod, cfg["spectrum"], cfg["edges"], cfg["patch_n"], N,
                         cfg["kappa"], [(0, 0), (77, 31)], K_TOL)
    # translation invariance across all nodes of every level (bands periodic on patches)
    for l in range(3):
        spread = np.abs(Kl[l] - Kl[l][0]).max() / np.abs(Kl[l][0]).max()
        assert spread < 1e-5, (l, spread)
    assert np.all(K[:, 0] > cfg["kappa"]) and np.all(K[:, 2] > cfg["kappa"])


def test_graph_replay_matches_direct_launches(mlsd, torch_mod, monkeypatch):
    # the captured CUDA graph of Algorithm 3 replays bit for bit what the direct
    # launches compute, on every replay
    spec = flows.continuous_spectrum(24, seed=5)
    args = (spec, 2e-3, 3, [1, 2, 4, 8, 16, 25], [32] * 5)
    dev = torch_mod.device("cuda:0")
    lv = mlsd.Levels(*args, n_burn_fixed=60, n_avg_fixed=40)
    K1 = torch_mod.zeros(9, 3, dtype=torch_mod.float64, device=dev)
    K2 = torch_mod.zeros_like(K1)
    lv.effective_diffusivity(K1)            # capture + replay
    lv.effective_diffusivity(K1)            # replay
    lv.effective_diffusivity(K2)            # new output pointer: capture again
    monkeypatch.setenv("MLSD_NO_GRAPH", "1")
    K3 = torch_mod.zeros_like(K1)
    lv.effective_diffusivity(K3)            # direct launches
    assert lv.status() == 0
    assert torch_mod.equal(K1, K2) and torch_mod.equal(K1, K3)


def test_chain_of_the_offdiagonal_stress_flow(mlsd, torch_mod):
    # the Sec. 4.3 structure at half the wavenumbers: two diagonal cellular
    # modes (2, 2) and (20, 20) and the off-diagonal pair (2, 18), (18, 2) of
    # level 1 (psi_12, psi_21), with patch sides 2 pi and pi; 64^2 patches on
    # level 2 (local wavenumber 10), reduced window
    spec = flows.cellular([(0.2, 2, 2), (0.2, 2, 18), (0.2, 18, 2), (0.2, 20, 20)])
    _chain_check(mlsd, torch_mod, spec, [1, 3, 21], [32, 64], 2, 1.0,
                 [(0, 0), (1, 1)], K_TOL, n_burn_fixed=150, n_avg_fixed=100, patch_div=[1, 2])


@pytest.mark.parametrize("periodize", [False, True])
def test_chain_on_side_2H_patches(mlsd, torch_mod, periodize):
    # the paper's local domains of side 2H (H = 2 pi / N): the bands are not
    # periodic on these patches; the seam is wrapped as sampled, or the band is
    # replaced by its periodic component (periodic-plus-smooth decomposition)
    N = 8
    spec = flows.cellular_two_scale(1.0, 0.5, 8)
    for pn in ([32, 32], [64, 32]):
        _chain_check(mlsd, torch_mod, spec, [1, 8, 9], pn, N, 0.05, [(0, 0), (3, 5), (7, 2)], K_TOL,
                     n_burn_fixed=200, n_avg_fixed=100, patch_div=[N // 2, 4 * N // 2],
                     periodize=periodize)


def test_periodize_rejects_what_it_does_not_support(mlsd, torch_mod):
    spec = flows.cellular_two_scale(1.0, 0.5, 8)
    for kw in (dict(patch_n=[128, 32]), dict(patch_n=[32, 32], precision="fp64")):
        pn = kw.pop("patch_n")
        with pytest.raises(mlsd.MlsdError):
            mlsd.Levels(spec, 0.05, 4, [1, 8, 9], pn, periodize=True, **kw)
