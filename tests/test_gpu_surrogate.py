"""GPU parity of the surrogate kernels against the oracle: patch features (DFT
and the perturbation moments of the steady corrector equation), the MLP
forward and gradient with bfloat16 rounding at the same points, and the
fallback path of the surrogate level solve."""
import math

import numpy as np
import pytest

import inputs
from inputs import flows
import oracle
from tests._parity import rel_l2

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


@pytest.mark.parametrize("n", [32, 64, 128, 256])
def test_features_match_oracle(mlsd, torch_mod, n):
    spec = flows.continuous_spectrum(40, seed=9)
    edges, N, kappa = [1, 4, 16, 41], 3, 2e-3
    lv = mlsd.Levels(spec, kappa, N, edges, [n, n, n], n_burn_fixed=1, n_avg_fixed=1)
    B = inputs.random_bases(N * N, kappa, 4)
    dev = torch_mod.device("cuda:0")
    Bd = torch_mod.tensor(B, dtype=torch_mod.float64, device=dev)
    X = torch_mod.zeros(N * N, mlsd.SUR_IN, dtype=torch_mod.bfloat16, device=dev)
    F = torch_mod.zeros(N * N, mlsd.SUR_FEATURES, dtype=torch_mod.float32, device=dev)
    lev, kind = oracle.band_of(spec, edges)
    for level in (2, 3):
        lv.features(level, Bd, X, F)
        torch_mod.cuda.synchronize()
        Fg = F.cpu().numpy()
        Nl = oracle.level_lattice(edges, [n] * 3)[level - 1]
        for p in range(N * N):
            ox = oracle.patch_origin(p % N, N, Nl, n); oy = oracle.patch_origin(p // N, N, Nl, n)
            psi = oracle.patch_psi(spec, Nl, ox, oy, n, use=(lev == level) & (kind == 0))
            f = oracle.features(psi, B[p], kappa)
            scale = np.abs(f[:578]).max()
            assert np.abs(Fg[p, :578] - f[:578]).max() < 1e-5 * scale, (level, p)
            np.testing.assert_allclose(Fg[p, 578:582], f[578:582], rtol=1e-6)
            # the moments T_2..T_6 (FP32 FFTs against the FP64 oracle), compared after
            # undoing the asinh: each to 1e-4 of itself, or 1e-5 of T_2's scale
            got, want = np.sinh(Fg[p, 582:606].astype(np.float64)), np.sinh(f[582:606])
            ts = np.abs(want[:3]).max()
            assert np.all(np.abs(got[:15] - want[:15]) <= 1e-4 * np.abs(want[:15]) + 1e-5 * ts), \
                (level, p, got, want)
            # the approximants: where the oracle's resummation has converged ([4/4]
            # within 1e-2 of [3/3]) they agree; where it has not (a Peclet number far
            # beyond the series' reach: Wynn's epsilon then amplifies the FP32
            # rounding of the moments up to T_19), both sides see it unconverged
            # and the fallback rule takes the patch
            q = psi
            if n > 64:                         # the features' 64 x 64 sub-lattice
                q = psi[::n // 64, ::n // 64]
                q = q - q.mean()
            T = oracle.series(q, B[p])
            _, _, E, gap = oracle.series_estimate(T)
            gp, ap = np.abs(got[21:24] - got[18:21]).max(), np.abs(got[21:24]).max()
            assert np.all(np.isfinite(got)), (level, p)
            if gap <= 1e-2 * np.abs(E).max():
                assert np.all(np.abs(got[15:] - want[15:]) <= 2e-3 * np.abs(want[15:]) + 1e-5 * ts), \
                    (level, p, got, want)
            else:
                assert gp > 1e-3 * ap, (level, p, got, want)
        # the bfloat16 row is the rounded FP32 row, zero padded
        Xg = X.float().cpu().numpy()
        nf = mlsd.SUR_FEATURES
        np.testing.assert_array_equal(Xg[:, :nf], F.to(torch_mod.bfloat16).float().cpu().numpy())
        assert not np.any(Xg[:, nf:])


@pytest.mark.parametrize("h,M", [(64, 96), (128, 777), (256, 2048)])
def test_gradient_matches_bf16_oracle(mlsd, torch_mod, h, M):
    # 96 rows: the short-k GEMMs run unsplit; 777 and 2048 rows (the training batch):
    # the weight-gradient GEMMs split k over CTAs, 777 with a ragged last split
    sur = mlsd.Surrogate(members=2, hidden=h, max_batch=M)
    rng = np.random.default_rng(5 + M)
    dev = torch_mod.device("cuda:0")
    for member in range(2):
        params = inputs.mlp_init(mlsd.SUR_IN, h, 100 + member) * 3.0
        params[::7] += 0.05                       # nonzero biases too
        sur.set_params(member, params)
        Xf = np.zeros((M, mlsd.SUR_IN), np.float32)
        nf = mlsd.SUR_FEATURES
        Xf[:, :nf] = rng.standard_normal((M, nf)).astype(np.float32)
        X = torch_mod.tensor(Xf, device=dev).to(torch_mod.bfloat16)
        Y = torch_mod.tensor(rng.standard_normal((M, 3)) * 0.3, dtype=torch_mod.float32, device=dev)
        g = torch_mod.zeros(sur.n_params, dtype=torch_mod.float32, device=dev)
        loss = sur.grad(member, X, Y, g)
        out_o, loss_o, g_o = oracle.mlp(X.float().cpu().numpy(), params.astype(np.float64), h,
                                        bf16=True, Y=Y.cpu().numpy(), want_grad=True)
        assert loss == pytest.approx(loss_o, rel=1e-4)
        g = g.cpu().numpy()
        # per tensor (W1 b1 W2 b2 W3 b3 W4 b4)
        sizes = [h * 640, h, h * h, h, h * h, h, 3 * h, 3]
        o = 0
        for sz in sizes:
            assert rel_l2(g[o:o + sz], g_o[o:o + sz]) < 1e-3, (member, o, sz)
            o += sz
        # prediction of every member equals the oracle forward
        out = torch_mod.zeros(2, M, 3, dtype=torch_mod.float32, device=dev)
        sur.predict(X, out)
        assert rel_l2(out[member].cpu().numpy(), out_o) < 1e-3


def test_training_lowers_the_loss(mlsd, torch_mod):
    # a smooth synthetic regression from the first features
    h, M = 64, 512
    sur = mlsd.Surrogate(members=1, hidden=h, max_batch=M)
    sur.set_params(0, inputs.mlp_init(mlsd.SUR_IN, h, 7))
    rng = np.random.default_rng(8)
    Xf = np.zeros((M, mlsd.SUR_IN), np.float32)
    Xf[:, :8] = rng.uniform(-1, 1, (M, 8))
    Yf = np.stack([np.sin(Xf[:, 0]), Xf[:, 1] * Xf[:, 2], 0.5 * Xf[:, 3] ** 2], 1).astype(np.float32)
    dev = torch_mod.device("cuda:0")
    X = torch_mod.tensor(Xf, device=dev).to(torch_mod.bfloat16)
    Y = torch_mod.tensor(Yf, device=dev)
    l0 = sur.train_step(0, X, Y, 2e-3, want_loss=True)
    for _ in range(300):
        sur.train_step(0, X, Y, 2e-3)
    l1 = sur.train_step(0, X, Y, 2e-3, want_loss=True)
    assert l1 < 0.1 * l0, (l0, l1)
    # parameters round-trip through the host (checkpoint / resume)
    p = sur.get_params(0)
    sur2 = mlsd.Surrogate(members=1, hidden=h, max_batch=M)
    sur2.set_params(0, p)
    o1 = torch_mod.zeros(1, M, 3, device=dev); o2 = torch_mod.zeros(1, M, 3, device=dev)
    sur.predict(X, o1); sur2.predict(X, o2)
    assert torch_mod.equal(o1, o2)


def test_library_training_loop_and_checkpoint(mlsd, torch_mod, tmp_path):
    # mlsd_surrogate_train (device gather of shuffled rows, Adam, geometric lr
    # decay) fits a smooth synthetic regression; the checkpoint file restores
    # the members bit for bit into a new handle
    h, n = 64, 1024
    sur = mlsd.Surrogate(members=2, hidden=h, max_batch=256)
    for m in range(2):
        sur.set_params(m, inputs.mlp_init(mlsd.SUR_IN, h, 17 + m))
    rng = np.random.default_rng(21)
    Xf = np.zeros((n, mlsd.SUR_IN), np.float32)
    Xf[:, :8] = rng.uniform(-1, 1, (n, 8))
    Yf = np.stack([np.sin(Xf[:, 0]), Xf[:, 1] * Xf[:, 2], 0.5 * Xf[:, 3] ** 2], 1).astype(np.float32)
    dev = torch_mod.device("cuda:0")
    X = torch_mod.tensor(Xf, device=dev).to(torch_mod.bfloat16)
    Y = torch_mod.tensor(Yf, device=dev)
    first = sur.train(X, Y, epochs=1, batch=128, lr=2e-3, seed=3)
    last = sur.train(X, Y, epochs=120, batch=128, lr=2e-3, lr_final=2e-4, seed=4)
    for m in range(2):
        assert last[m] < 0.3 * first[m], (first, last)
    path = tmp_path / "ensemble.bin"
    sur.save(path)
    sur2 = mlsd.Surrogate(members=2, hidden=h, max_batch=256)
    sur2.load(path)
    for m in range(2):
        assert np.array_equal(sur.get_params(m), sur2.get_params(m))
    o1 = torch_mod.zeros(2, n, 3, device=dev); o2 = torch_mod.zeros(2, n, 3, device=dev)
    sur.predict(X, o1); sur2.predict(X, o2)
    assert torch_mod.equal(o1, o2)
    # a file of another shape is refused
    with pytest.raises(mlsd.MlsdError):
        mlsd.Surrogate(members=3, hidden=h, max_batch=256).load(path)


@pytest.mark.parametrize("n", [32, 128])
def test_surrogate_level_fallback_paths(mlsd, torch_mod, n):
    # n = 128: features on the 64 x 64 sub-lattice, fallback solves by the cluster kernel
    spec = flows.continuous_spectrum(40, seed=9)
    edges, N, kappa = [1, 4, 16, 41], 4, 2e-3
    lv = mlsd.Levels(spec, kappa, N, edges, [n] * 3, n_burn_fixed=50, n_avg_fixed=50)
    dev = torch_mod.device("cuda:0")
    B = torch_mod.tensor(inputs.random_bases(N * N, kappa, 1), dtype=torch_mod.float64, device=dev)
    K_plain = torch_mod.zeros_like(B)
    lv.solve_level(2, B, K_plain)
    sur = mlsd.Surrogate(members=4, hidden=64, max_batch=64)
    for m in range(4):
        sur.set_params(m, inputs.mlp_init(mlsd.SUR_IN, 64, m))
    # threshold 0: every patch falls back -> the plain result (a few fallback patches
    # run the lowest-latency tiling, so only the order of the flux sums may differ)
    K0 = torch_mod.zeros_like(B)
    assert lv.solve_level_surrogate(sur, 2, B, K0, 0.0) == N * N
    assert rel_l2(K0.cpu().numpy(), K_plain.cpu().numpy()) < 1e-6
    # huge threshold: no fallback, K = B + E + tr(B) * ensemble mean / Y_SCALE
    K1 = torch_mod.zeros_like(B)
    assert lv.solve_level_surrogate(sur, 2, B, K1, 1e30) == 0
    X = torch_mod.zeros(N * N, mlsd.SUR_IN, dtype=torch_mod.bfloat16, device=dev)
    F = torch_mod.zeros(N * N, mlsd.SUR_FEATURES, dtype=torch_mod.float32, device=dev)
    lv.features(2, B, X, F)
    out = torch_mod.zeros(4, N * N, 3, device=dev)
    sur.predict(X, out)
    tr = (B[:, 0] + B[:, 2]).unsqueeze(1)
    E = torch_mod.sinh(F[:, 603:606].double()) * tr / mlsd.SUR_T_SCALE   # FP32-rounded copy of E
    want = B + E + tr * torch_mod.sinh(out.double()).mean(0) / mlsd.SUR_Y_SCALE
    assert rel_l2(K1.cpu().numpy(), want.cpu().numpy()) < 1e-6
    assert torch_mod.allclose(K1, want, rtol=1e-6, atol=0)
    assert lv.status() == 0


@pytest.mark.parametrize("tma", [True, False])
@pytest.mark.parametrize("M,h", [(300, 256), (128, 64), (1000, 128), (4099, 256), (20000, 256)])
def test_tensor_core_inference_matches_oracle(mlsd, torch_mod, M, h, tma, monkeypatch):
    # tcgen05 engine (TMA-fed ring, or the thread-staged fallback) against the
    # bfloat16-emulating oracle and the CUDA-core engine
    if not tma:
        monkeypatch.setenv("MLSD_NO_TMA", "1")
    members = 2
    # the CUDA-core engine runs in chunks of max_batch rows; the largest case is one
    # chunk big enough for its GEMMs to take the 128-wide tiles
    sur = mlsd.Surrogate(members=members, hidden=h, max_batch=M if M >= 20000 else 512)
    rng = np.random.default_rng(M + h)
    params = []
    for m in range(members):
        p = inputs.mlp_init(mlsd.SUR_IN, h, 40 + m) * 2.0
        o = h * mlsd.SUR_IN
        p[o:o + h] = rng.uniform(-0.2, 0.2, h)            # biases of layer 1
        params.append(p)
        sur.set_params(m, p)
    dev = torch_mod.device("cuda:0")
    Xf = np.zeros((M, mlsd.SUR_IN), np.float32)
    Xf[:, :mlsd.SUR_FEATURES] = rng.standard_normal((M, mlsd.SUR_FEATURES))
    X = torch_mod.tensor(Xf, device=dev).to(torch_mod.bfloat16)
    out_tc = torch_mod.full((members, M, 3), float("nan"), device=dev)
    sur.set_engine(mlsd.SUR_TENSOR)
    sur.predict(X, out_tc)
    assert sur.status() == 0
    out_cc = torch_mod.zeros(members, M, 3, device=dev)
    sur.set_engine(mlsd.SUR_CUDA)
    sur.predict(X, out_cc)
    Xo = X.float().cpu().numpy()
    rows = np.r_[0:min(M, 400), max(0, M - 200):M]          # the oracle on a sample of rows
    Xo = Xo[rows]
    out_tc = out_tc[:, rows]
    out_cc = out_cc[:, rows]
    for m in range(members):
        ref = oracle.mlp(Xo, params[m].astype(np.float64), h, bf16=True)
        assert rel_l2(out_tc[m].cpu().numpy(), ref) < 1e-3, m
        assert rel_l2(out_cc[m].cpu().numpy(), ref) < 1e-3, m


def _octave_band(seed, lo, hi):
    full = flows.continuous_spectrum(256, seed=seed)
    a, b = np.abs(full.k1), np.abs(full.k2)
    keep = (a >= lo) & (a < hi) & (b >= lo) & (b < hi)
    return flows.Spectrum(full.k1[keep], full.k2[keep], full.re[keep], full.im[keep])


def test_trained_surrogate_replaces_most_patch_solves(mlsd, torch_mod):
    # What the learned part gains over the method without it: trained on the
    # library's own plain solves of one flow realization's 5th-octave band (64^2
    # patches, the highest Peclet numbers of the surrogate's levels; 2 base sets),
    # the ensemble answers the patches of ANOTHER realization (no psi seen in
    # training) with a fresh base set; only the patches it is unsure of are solved
    # again, and the answers stay within 1e-3 of the plain solve.  Without the
    # network (zero weights: K = B + E, the resummed series) fewer patches are
    # within 1e-3.
    from paper_1510_00451_gb300 import surrogate as S
    N, kappa = 128, 1e-3
    P = N * N
    lv = mlsd.Levels(_octave_band(1510004510, 16, 32), kappa, N, [16.0, 32.0], [64],
                     patch_div=[16], cfl=0.2)
    X, Y = S.make_dataset(lv, 1, [inputs.random_bases(P, kappa, 70 + i) for i in range(2)])
    lv.close()
    sur = mlsd.Surrogate(members=4, hidden=128, max_batch=1024)
    for m in range(4):
        sur.set_params(m, inputs.mlp_init(mlsd.SUR_IN, 128, 90 + m))
    losses = sur.train(X, Y, epochs=80, batch=1024, lr=3e-3, seed=1, lr_final=1e-5)
    assert max(losses) < 0.02                   # asinh targets; the accuracy is checked below
    lt = mlsd.Levels(_octave_band(77, 16, 32), kappa, N, [16.0, 32.0], [64], patch_div=[16],
                     cfl=0.2)
    dev = torch_mod.device("cuda:0")
    Bt = torch_mod.tensor(inputs.random_bases(P, kappa, 99), dtype=torch_mod.float64, device=dev)
    K_plain = torch_mod.zeros_like(Bt)
    lt.solve_level(1, Bt, K_plain)
    K_sur = torch_mod.zeros_like(Bt)
    n_fb = lt.solve_level_surrogate(sur, 1, Bt, K_sur, 1e-3)
    assert lt.status() == 0 and sur.status() == 0
    err = S.k_error(K_sur.cpu().numpy(), K_plain.cpu().numpy())
    assert n_fb < P // 5, n_fb                  # most patch solves are replaced
    assert np.median(err) < 1e-4, np.median(err)
    assert np.quantile(err, 0.99) <= 1e-3, np.quantile(err, 0.99)
    K_net = torch_mod.zeros_like(Bt)
    lt.solve_level_surrogate(sur, 1, Bt, K_net, 1e30)
    sur0 = mlsd.Surrogate(members=4, hidden=128, max_batch=1024)    # zero weights: K = B + E
    K_ser = torch_mod.zeros_like(Bt)
    lt.solve_level_surrogate(sur0, 1, Bt, K_ser, 1e30)
    e_net = S.k_error(K_net.cpu().numpy(), K_plain.cpu().numpy())
    e_ser = S.k_error(K_ser.cpu().numpy(), K_plain.cpu().numpy())
    assert np.mean(e_net <= 1e-3) > np.mean(e_ser <= 1e-3) + 0.005, \
        (np.mean(e_net <= 1e-3), np.mean(e_ser <= 1e-3))


@pytest.mark.parametrize("n", [32, 128])
def test_chain_in_surrogate_mode(mlsd, torch_mod, n):
    # Algorithm 3 with a surrogate attached to the finest level: at threshold 0
    # every patch falls back and the chain equals the plain chain; at a huge
    # threshold the finest K* is the ensemble's and the coarser level is solved
    # on it as on any base (n = 128: the finest level's fallback runs the cluster
    # kernel, sized on the device inside the captured chain)
    spec = flows.cellular_two_scale(1.0, 0.4, 8)
    N, kappa = 4, 0.05
    lv = mlsd.Levels(spec, kappa, N, [1, 8, 16], [32, n], n_burn_fixed=120, n_avg_fixed=80)
    dev = torch_mod.device("cuda:0")
    P = N * N
    K_plain = torch_mod.zeros(P, 3, dtype=torch_mod.float64, device=dev)
    KL_plain = torch_mod.zeros(2, P, 3, dtype=torch_mod.float64, device=dev)
    lv.effective_diffusivity(K_plain, KL_plain)
    sur = mlsd.Surrogate(members=2, hidden=64, max_batch=64)
    for m in range(2):
        sur.set_params(m, inputs.mlp_init(mlsd.SUR_IN, 64, 5 + m))
    with pytest.raises(mlsd.MlsdError):                 # no surrogate attached yet
        lv.effective_diffusivity(K_plain.clone(), mode=mlsd.MLSD_SURROGATE)
    lv.attach_surrogate(2, sur, 0.0)
    K0 = torch_mod.zeros_like(K_plain)
    lv.effective_diffusivity(K0, mode=mlsd.MLSD_SURROGATE)
    assert lv.status() == 0 and lv.surrogate_fallbacks(2) == P
    assert rel_l2(K0.cpu().numpy(), K_plain.cpu().numpy()) < 1e-6
    lv.attach_surrogate(2, sur, 1e30)
    K1 = torch_mod.zeros_like(K_plain)
    KL1 = torch_mod.zeros_like(KL_plain)
    lv.effective_diffusivity(K1, KL1, mode=mlsd.MLSD_SURROGATE)
    assert lv.status() == 0 and lv.surrogate_fallbacks(2) == 0
    # finest level: no off-diagonal parts, so its base is kappa I
    Bf = torch_mod.tensor(np.tile([kappa, 0.0, kappa], (P, 1)), dtype=torch_mod.float64, device=dev)
    Ks = torch_mod.zeros_like(Bf)
    lv.solve_level_surrogate(sur, 2, Bf, Ks, 1e30)
    assert torch_mod.allclose(KL1[1], Ks, rtol=1e-12, atol=0)
    # coarse level on that base, solved plainly (the chain's base is K* - B + B,
    # equal to K* up to FP64 rounding, which can move the FP32 coefficients)
    Kc = torch_mod.zeros_like(Bf)
    lv.solve_level(1, Ks, Kc)
    assert rel_l2(K1.cpu().numpy(), Kc.cpu().numpy()) < 1e-6
    lv.attach_surrogate(2, None, 0.0)
    K2 = torch_mod.zeros_like(K_plain)
    lv.effective_diffusivity(K2)                        # plain chain again (graph replay)
    assert torch_mod.equal(K2, K_plain)


def _oracle_target(K, B, psi):
    _, _, E, _ = oracle.series_estimate(oracle.series(psi, B))
    return oracle.surrogate_target(K, B, E)


def test_dataset_targets_match_oracle(mlsd, torch_mod):
    # mlsd_surrogate_dataset: Y = asinh((K - B - E) 300 / tr(B)) from the library's
    # own plain solves and series, against the oracle's
    from tests._parity import oracle_level
    spec = flows.continuous_spectrum(40, seed=9)
    edges, N, kappa, n = [1, 4, 16, 41], 3, 2e-3, 32
    lv = mlsd.Levels(spec, kappa, N, edges, [n, n, n], n_burn_fixed=60, n_avg_fixed=40)
    P = N * N
    B = inputs.random_bases(P, kappa, 12)
    dev = torch_mod.device("cuda:0")
    Bd = torch_mod.tensor(B, dtype=torch_mod.float64, device=dev)
    X = torch_mod.zeros(P, mlsd.SUR_IN, dtype=torch_mod.bfloat16, device=dev)
    Y = torch_mod.zeros(P, 3, dtype=torch_mod.float32, device=dev)
    lv.surrogate_dataset(3, Bd, X, Y)
    assert lv.status() == 0
    Yg = Y.cpu().numpy()
    Kr = oracle_level(spec, edges, [n] * 3, 3, N, B, list(range(P)), n_burn_fixed=60, n_avg_fixed=40)
    lev, kind = oracle.band_of(spec, edges)
    Nl = oracle.level_lattice(edges, [n] * 3)[2]
    for p in range(P):
        ox = oracle.patch_origin(p % N, N, Nl, n); oy = oracle.patch_origin(p // N, N, Nl, n)
        psi = oracle.patch_psi(spec, Nl, ox, oy, n, use=(lev == 3) & (kind == 0))
        tr = B[p, 0] + B[p, 2]
        want = _oracle_target(Kr[p], B[p], psi)
        # in K units: sinh(Y) tr / 300 against the oracle's, to 1e-5 of K
        dk = np.abs(np.sinh(Yg[p].astype(np.float64)) - np.sinh(want)) * tr / mlsd.SUR_Y_SCALE
        assert dk.max() < 1e-5 * np.abs(Kr[p]).max(), (p, Yg[p], want)
    assert np.abs(Yg).max() > 1e-3                      # targets are not all zero


@pytest.mark.parametrize("g", range(8))
def test_symmetry_images_match_the_oracle(mlsd, torch_mod, g):
    # mlsd_surrogate_symmetry on the library's own dataset rows: the image under
    # element g of the square's group against the oracle's features and target
    # of the mapped patch (psi mapped on the grid, base R B R^T, its own solve)
    from tests._parity import level_geometry, square_symmetry_psi, square_symmetry_tensor
    spec = flows.continuous_spectrum(40, seed=9)
    edges, N, kappa, n, nb, na = [1, 4, 16, 41], 3, 2e-3, 32, 60, 40
    lv = mlsd.Levels(spec, kappa, N, edges, [n, n, n], n_burn_fixed=nb, n_avg_fixed=na)
    P = N * N
    B = inputs.random_bases(P, kappa, 12)
    dev = torch_mod.device("cuda:0")
    Bd = torch_mod.tensor(B, dtype=torch_mod.float64, device=dev)
    X = torch_mod.zeros(P, mlsd.SUR_IN, dtype=torch_mod.bfloat16, device=dev)
    Y = torch_mod.zeros(P, 3, dtype=torch_mod.float32, device=dev)
    lv.surrogate_dataset(3, Bd, X, Y)
    Xg = torch_mod.full_like(X, float("nan"))
    Yg = torch_mod.full_like(Y, float("nan"))
    mlsd.surrogate_symmetry(X, Y, g, Xg, Yg)
    torch_mod.cuda.synchronize()
    assert lv.status() == 0
    Xn = Xg.float().cpu().numpy()
    Yn = Yg.cpu().numpy()
    lev, kind = oracle.band_of(spec, edges)
    _, Nl, h, _ = level_geometry(edges, [n] * 3, 3)
    for p in range(P):
        ox = oracle.patch_origin(p % N, N, Nl, n); oy = oracle.patch_origin(p // N, N, Nl, n)
        psi = square_symmetry_psi(oracle.patch_psi(spec, Nl, ox, oy, n, use=(lev == 3) & (kind == 0)), g)
        Bg = square_symmetry_tensor(B[p], g)
        f = oracle.features(psi, Bg, kappa)
        # bfloat16 rows: the FP32 features (1e-5 of each group's scale) rounded to 8 bits
        for lo, hi, tol in ((0, 578, 2e-5), (578, 582, 1e-6), (582, 606, 2e-5)):
            d = np.abs(Xn[p, lo:hi] - f[lo:hi])
            assert np.all(d <= 2.0 ** -8 * np.abs(f[lo:hi]) + tol * np.abs(f[lo:hi]).max()), (g, p, lo)
        assert not np.any(Xn[p, mlsd.SUR_FEATURES:])
        v1, v2 = oracle.velocity(psi, h)
        dt = oracle.micro_dt(h, float(np.max(np.abs(v1) + np.abs(v2))), Bg, 0.2)
        Kg = oracle.patch_k(psi, h, Bg, dt, nb, na)
        tr = Bg[0] + Bg[2]
        want = _oracle_target(Kg, Bg, psi)
        dk = np.abs(np.sinh(Yn[p].astype(np.float64)) - np.sinh(want)) * tr / mlsd.SUR_Y_SCALE
        assert dk.max() < 1e-5 * np.abs(Kg).max(), (g, p, Yn[p], want)


def test_augmented_training_is_deterministic_and_learns(mlsd, torch_mod):
    # mlsd_surrogate_train with augment: every row enters with its 8 images; on
    # an equivariant regression (the matrix square of B / kappa, a tensor) the
    # loss drops, and one seed gives the same parameters twice
    h, n = 64, 512
    rng = np.random.default_rng(8)
    Xf = np.zeros((n, mlsd.SUR_IN), np.float32)
    a = rng.uniform(0.5, 2.0, (n, 2))
    c = rng.uniform(-0.5, 0.5, n) * np.sqrt(a[:, 0] * a[:, 1])
    Xf[:, 578], Xf[:, 579], Xf[:, 580] = a[:, 0], c, a[:, 1]
    Xf[:, 581] = math.log(1e-3)
    Yf = 0.2 * np.stack([a[:, 0] ** 2 + c ** 2, c * (a[:, 0] + a[:, 1]), a[:, 1] ** 2 + c ** 2], 1)
    dev = torch_mod.device("cuda:0")
    X = torch_mod.tensor(Xf, device=dev).to(torch_mod.bfloat16)
    Y = torch_mod.tensor(Yf.astype(np.float32), device=dev)
    runs = []
    for _ in range(2):
        sur = mlsd.Surrogate(members=1, hidden=h, max_batch=256)
        sur.set_params(0, inputs.mlp_init(mlsd.SUR_IN, h, 5))
        first = sur.train(X, Y, epochs=1, batch=256, lr=2e-3, seed=7, augment=True)
        last = sur.train(X, Y, epochs=40, batch=256, lr=2e-3, lr_final=2e-4, seed=8, augment=True)
        assert last[0] < 0.3 * first[0], (first, last)
        runs.append(sur.get_params(0))
    assert np.array_equal(runs[0], runs[1])


def test_surrogate_chain_replays_as_a_graph(mlsd, torch_mod, monkeypatch):
    # MLSD_SURROGATE chains run as one captured CUDA graph: the fallback solve is
    # launched for every patch and reads the fallback count on the device, so no
    # step needs the host (a host synchronisation inside the capture would fail
    # it).  The replays equal the chain launched directly, with the same count;
    # with every patch falling back the chain is the plain one.
    spec = flows.combine(flows.cellular_two_scale(1.0, 0.4, 8), flows.continuous_spectrum(12, seed=3))
    N, kappa = 6, 0.05
    lv = mlsd.Levels(spec, kappa, N, [1, 8, 16], [32, 32], n_burn_fixed=60, n_avg_fixed=40)
    dev = torch_mod.device("cuda:0")
    P = N * N
    K_plain = torch_mod.zeros(P, 3, dtype=torch_mod.float64, device=dev)
    lv.effective_diffusivity(K_plain)
    sur = mlsd.Surrogate(members=2, hidden=64, max_batch=64)
    for m in range(2):
        sur.set_params(m, inputs.mlp_init(mlsd.SUR_IN, 64, 11 + m) * (0.05 if m == 0 else 2.0))
    for thr in (0.0, 2e-3, 1e30):
        monkeypatch.delenv("MLSD_NO_GRAPH", raising=False)
        lv.attach_surrogate(2, sur, thr)
        K1 = torch_mod.zeros(P, 3, dtype=torch_mod.float64, device=dev)
        lv.effective_diffusivity(K1, mode=mlsd.MLSD_SURROGATE)          # capture + replay
        n1 = lv.surrogate_fallbacks(2)
        K1b = torch_mod.zeros_like(K1)
        lv.effective_diffusivity(K1b, mode=mlsd.MLSD_SURROGATE)         # new output: capture again
        lv.effective_diffusivity(K1b, mode=mlsd.MLSD_SURROGATE)         # replay
        assert lv.status() == 0 and sur.status() == 0
        monkeypatch.setenv("MLSD_NO_GRAPH", "1")
        K2 = torch_mod.zeros_like(K1)
        lv.effective_diffusivity(K2, mode=mlsd.MLSD_SURROGATE)
        assert lv.surrogate_fallbacks(2) == n1
        assert torch_mod.equal(K1, K1b) and torch_mod.equal(K1, K2), thr
        if thr == 0.0:
            assert n1 == P
            assert rel_l2(K1.cpu().numpy(), K_plain.cpu().numpy()) < 1e-6
        if thr == 1e30:
            assert n1 == 0
