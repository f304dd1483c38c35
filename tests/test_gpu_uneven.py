"""Uneven patch sizes within a level: the patch-size rule and the chain with
mixed 32^2 ... 256^2 patches (size classes launched concurrently, or every
patch of a level in one persistent launch) against the oracle with the same
per-node sizes."""
import numpy as np
import pytest

from inputs import flows
import oracle
from tests._parity import oracle_level, rel_l2

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def problem():
    spec = flows.continuous_spectrum(48, seed=5)
    return dict(spec=spec, edges=[1, 2, 4, 8, 16, 32, 49], N=3, kappa=2e-3)


def test_patch_size_rule_matches_oracle(problem):
    import paper_1510_00451_gb300 as mlsd
    pr = problem
    L = len(pr["edges"]) - 1
    lv = mlsd.Levels(pr["spec"], pr["kappa"], pr["N"], pr["edges"], [0] * L,
                     n_burn_fixed=1, n_avg_fixed=1)
    seen = set()
    for l in range(1, L + 1):
        got = lv.patch_sizes(l)
        for p in range(pr["N"] ** 2):
            n, _ = oracle.patch_n_rule(pr["spec"], pr["edges"], l, (p % pr["N"], p // pr["N"]),
                                       pr["N"], pr["kappa"])
            assert got[p] == n, (l, p, got[p], n)
            seen.add(int(n))
    assert len(seen) >= 3          # the workload really is uneven


def test_uneven_chain_parity(problem):
    import torch
    import paper_1510_00451_gb300 as mlsd
    pr = problem
    L = len(pr["edges"]) - 1
    N = pr["N"]
    lv = mlsd.Levels(pr["spec"], pr["kappa"], N, pr["edges"], [0] * L,
                     n_burn_fixed=60, n_avg_fixed=40)
    sizes = np.stack([lv.patch_sizes(l + 1) for l in range(L)], 1)      # [P][L]
    mixed = [l for l in range(L) if len(set(sizes[:, l])) > 1]
    K = torch.zeros(N * N, 3, dtype=torch.float64, device="cuda:0")
    lv.effective_diffusivity(K)
    assert lv.status() == 0
    K = K.cpu().numpy()
    nodes = [(p % N, p // N) for p in range(N * N)]
    want = oracle.chain(pr["spec"], pr["edges"], [32] * L, N, pr["kappa"], nodes,
                        n_burn_fixed=60, n_avg_fixed=40, node_n=sizes)
    for p in range(N * N):
        assert rel_l2(K[p], want[p]) < 1e-4, (p, K[p], want[p])
    info = [lv.info(l + 1) for l in range(L)]
    assert max(i["n_classes"] for i in info) >= 1
    print("levels with mixed sizes:", mixed, [i["n"] for i in info])


def test_explicit_size_map_parity():
    import torch
    import paper_1510_00451_gb300 as mlsd
    spec = flows.cellular_hierarchy(2, 4)
    edges, N, kappa = [1, 4, 16], 4, 0.02
    P = N * N
    rng = np.random.default_rng(3)
    nmap = rng.choice([32, 64], size=(2, P)).astype(np.int32)      # [L][P]
    lv = mlsd.Levels(spec, kappa, N, edges, [0, 0], patch_n_map=nmap,
                     n_burn_fixed=80, n_avg_fixed=60)
    assert lv.info(1)["n_classes"] == 2 and lv.info(2)["n_classes"] == 2
    K = torch.zeros(P, 3, dtype=torch.float64, device="cuda:0")
    lv.effective_diffusivity(K)
    assert lv.status() == 0
    K = K.cpu().numpy()
    nodes = [(p % N, p // N) for p in range(P)]
    want = oracle.chain(spec, edges, [32, 32], N, kappa, nodes, n_burn_fixed=80, n_avg_fixed=60,
                        node_n=nmap.T)
    for p in range(P):
        assert rel_l2(K[p], want[p]) < 1e-4
    # the work count follows the per-patch sizes
    cu, ms, wu = lv.level_work(1)
    assert cu == sum(2 * int(n) ** 2 * 140 for n in nmap[0])
    assert wu == sum(2 * int(n) ** 2 * 60 for n in nmap[0])
    assert ms == 140


@pytest.mark.slow
def test_full_size_continuous_spectrum_sampled_patches():
    # the continuous-spectrum hierarchy at full size (8 octave levels, 256 x 256 macro
    # nodes, 32^2 .. 256^2 patches from the size rule), every level solved on seeded
    # full-tensor bases with the bench's 32-step window; sampled patches of every
    # level and size class against the oracle's patch solve (w and K)
    import torch
    import inputs
    import paper_1510_00451_gb300 as mlsd
    from tests._parity import oracle_level
    cfg = inputs.config_problem("continuous_spectrum")
    N, L, kappa = cfg["n_macro"], len(cfg["edges"]) - 1, cfg["kappa"]
    P = N * N
    lv = mlsd.Levels(cfg["spectrum"], kappa, N, cfg["edges"], [0] * L, cfl=cfg["cfl"],
                     n_burn_fixed=0, n_avg_fixed=32)
    rng = np.random.default_rng(1510)
    dev = torch.device("cuda:0")
    for level in range(1, L + 1):
        sizes = lv.patch_sizes(level)
        B = inputs.random_bases(P, kappa, 2000 + level)
        Bd = torch.tensor(B, dtype=torch.float64, device=dev)
        K = torch.zeros_like(Bd)
        lv.solve_level(level, Bd, K)
        assert lv.status() == 0
        K = K.cpu().numpy()
        assert np.isfinite(K).all()
        for n in sorted(set(int(v) for v in sizes)):
            cand = np.flatnonzero(sizes == n)
            picks = rng.choice(cand, size=min(3, len(cand)), replace=False)
            pn = [32] * L
            pn[level - 1] = n
            ref = oracle_level(cfg["spectrum"], cfg["edges"], pn, level, N, B, list(picks),
                               cfl=cfg["cfl"], n_burn_fixed=0, n_avg_fixed=32)
            for p, Kr in zip(picks, ref):
                assert rel_l2(K[p], Kr) < 1e-4, (level, n, p, K[p], Kr)


@pytest.mark.slow
def test_full_size_continuous_spectrum_chain_at_sampled_nodes():
    # Algorithm 3 down all 8 octave levels of the full continuous spectrum
    # (|k| <= 256, ~1e5 modes, 256 x 256 macro nodes, 32^2 .. 256^2 patches from
    # the size rule, off-diagonal closed forms included), every node solved on
    # the GPU with a fixed 32-step window; the composed K at sampled nodes
    # against the oracle's chain at those nodes with the same per-level sizes
    import torch
    import paper_1510_00451_gb300 as mlsd
    from inputs import flows as fl
    cfg = fl.config_problem("continuous_spectrum")
    N, L, kappa = cfg["n_macro"], len(cfg["edges"]) - 1, cfg["kappa"]
    lv = mlsd.Levels(cfg["spectrum"], kappa, N, cfg["edges"], [0] * L, cfl=cfg["cfl"],
                     n_burn_fixed=0, n_avg_fixed=32)
    sizes = np.stack([lv.patch_sizes(l + 1) for l in range(L)], 1)      # [P][L]
    K = torch.zeros(N * N, 3, dtype=torch.float64, device="cuda:0")
    lv.effective_diffusivity(K)
    assert lv.status() == 0
    K = K.cpu().numpy()
    assert np.isfinite(K).all()
    rng = np.random.default_rng(20261204)
    picks = rng.choice(N * N, size=2, replace=False)
    for p in picks:
        # one node per call: the oracle's threads then split that node's line variances
        Kr = oracle.chain(cfg["spectrum"], cfg["edges"], [32] * L, N, kappa,
                          [(int(p) % N, int(p) // N)], cfl=cfg["cfl"], n_burn_fixed=0,
                          n_avg_fixed=32, node_n=sizes[[p]])[0]
        assert rel_l2(K[p], Kr) < 1e-4, (int(p), sizes[p], K[p], Kr)


def test_profile_by_patch_size(problem):
    # profiling mode 2 runs a level's sizes one after another: the same K bit for bit
    # as the concurrent launches, and one timing entry per patch size of each level
    import torch
    import paper_1510_00451_gb300 as mlsd
    pr = problem
    L = len(pr["edges"]) - 1
    N = pr["N"]
    lv = mlsd.Levels(pr["spec"], pr["kappa"], N, pr["edges"], [0] * L,
                     n_burn_fixed=20, n_avg_fixed=10)
    K = torch.zeros(N * N, 3, dtype=torch.float64, device="cuda:0")
    lv.effective_diffusivity(K)
    K0 = K.clone()
    for l in range(L):
        lv.profile_collect_classes(l + 1)
    lv.profile(True, serial_classes=True)
    lv.effective_diffusivity(K)
    torch.cuda.synchronize()
    lv.profile(False)
    assert lv.status() == 0
    assert torch.equal(K, K0)
    for l in range(L):
        cls = lv.profile_collect_classes(l + 1)
        if lv.info(l + 1)["level_launch"]:
            assert set(cls) == {0}
        else:
            assert set(cls) == set(int(n) for n in lv.patch_sizes(l + 1))
        assert all(ms > 0 and n == 1 for ms, n in cls.values())


@pytest.mark.parametrize("mode", [1, 2])
def test_uneven_chain_parity_one_launch(problem, monkeypatch, mode):
    # every mixed-size level in one persistent launch (forced; schedule 1: 256^2
    # fields first, 2: interleaved), against the oracle with the same per-node sizes
    import torch
    import paper_1510_00451_gb300 as mlsd
    monkeypatch.setenv("MLSD_LEVEL", str(mode))
    pr = problem
    L = len(pr["edges"]) - 1
    N = pr["N"]
    lv = mlsd.Levels(pr["spec"], pr["kappa"], N, pr["edges"], [0] * L,
                     n_burn_fixed=60, n_avg_fixed=40)
    sizes = np.stack([lv.patch_sizes(l + 1) for l in range(L)], 1)      # [P][L]
    mixed = [l for l in range(L) if len(set(sizes[:, l])) > 1]
    assert mixed
    for l in range(L):
        assert lv.info(l + 1)["level_launch"] == (mode if l in mixed else 0)
    K = torch.zeros(N * N, 3, dtype=torch.float64, device="cuda:0")
    lv.effective_diffusivity(K)
    assert lv.status() == 0
    K = K.cpu().numpy()
    nodes = [(p % N, p // N) for p in range(N * N)]
    want = oracle.chain(pr["spec"], pr["edges"], [32] * L, N, pr["kappa"], nodes,
                        n_burn_fixed=60, n_avg_fixed=40, node_n=sizes)
    for p in range(N * N):
        assert rel_l2(K[p], want[p]) < 1e-4, (p, K[p], want[p])


def _all_sizes_level(monkeypatch, mode):
    import torch
    import paper_1510_00451_gb300 as mlsd
    monkeypatch.setenv("MLSD_LEVEL", str(mode))
    spec = flows.cellular_two_scale(0.8, 0.5, 4)
    edges, N, kappa = [1, 4, 8], 5, 0.03
    P = N * N
    nmap = np.full((2, P), 32, dtype=np.int32)
    nmap[1] = np.array([32, 64, 128, 256, 64, 32, 128, 32, 64, 256, 32, 64, 128, 32, 32,
                        64, 32, 128, 64, 32, 256, 32, 64, 32, 128], dtype=np.int32)
    lv = mlsd.Levels(spec, kappa, N, edges, [0, 0], patch_n_map=nmap,
                     n_burn_fixed=40, n_avg_fixed=30)
    assert lv.info(2)["n_classes"] == 4 and lv.info(2)["level_launch"] == mode
    B = np.tile([kappa * 1.3, 0.2 * kappa, kappa * 0.9], (P, 1))
    dev = torch.device("cuda:0")
    Kb = torch.tensor(B, dtype=torch.float64, device=dev)
    Ko = torch.zeros_like(Kb)
    lv.solve_level(2, Kb, Ko)
    assert lv.status() == 0
    return nmap, B, Ko.cpu().numpy(), spec, edges, N, kappa


@pytest.mark.parametrize("mode", [1, 2])
def test_one_launch_level_of_all_four_sizes(monkeypatch, mode):
    # a level mixing 32^2, 64^2, 128^2 and 256^2 patches in one launch: the K of the
    # per-size launches up to the FP32 grouping of the flux sums (the cells'
    # arithmetic is the same, but a thread's block of cells, over which it sums
    # in FP32, may have another shape in the tiling the tuner picked for a size),
    # and K against the oracle for one patch of each size
    nmap, B, K1, spec, edges, N, kappa = _all_sizes_level(monkeypatch, mode)
    _, _, K0, *_ = _all_sizes_level(monkeypatch, 0)
    for p in range(N * N):
        assert rel_l2(K1[p], K0[p]) < 1e-6, (p, nmap[1, p], K1[p], K0[p])
    for p in (0, 1, 2, 3):
        Kr = oracle_level(spec, edges, [32, int(nmap[1, p])], 2, N, B, [p],
                          n_burn_fixed=40, n_avg_fixed=30)[0]
        assert rel_l2(K1[p], Kr) < 1e-4, (p, K1[p], Kr)
