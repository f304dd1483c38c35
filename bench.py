#!/usr/bin/env python3
"""Throughput benchmark of the batched multiscale effective-diffusivity solve.

One step = the whole hot path on the 3-level cellular hierarchy
(psi = sum_j 4^-j sin(4^j x) sin(4^j y), kappa = 0.01, 128 x 128 macro grid,
one 64^2 patch per macro node and level, 16384 patches per level, FP32 stencil
with FP64 averages, full relaxation window): Algorithm 3 over the 3 levels
(off-diagonal closed forms, three levels of batched patch solves, composition)
followed by the macro solve of U_t = div(K grad U) to T = 1.

Printed (rank 0, one JSON line): patch cell-updates/s of the whole job (a
cell-update = one cell of one corrector field advanced one full RK2 step),
K_eff tensors/s, the roofline of the patch-solve kernel, the oracle timed on
the host cores, an end-to-end figure through the C ABI with host buffers, SM
clocks sampled during the timed region, and the number of library kernel
launches inside it.

--impl reference times the FP64 CPU oracle on a bounded sample of the same
workload (there is no other implementation of this method to compare with).
"""
import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

METRIC = "K_eff tensors/s & patch cell-updates/s, surrogate vs plain GPU at ≤1e-3 K_eff err"
UNIT = "cell-updates/s"
# Algorithmic FP32 work of k_patch_solve.  Per cell-update (one cell of one field,
# one full Heun step): stage 1 = 4 FADD + 6 FFMA, stage 2 = 4 FADD + 7 FFMA.
# Per cell-update inside the averaging window, add the flux sums: 2 FFMA + 1 FADD.
OPS_PER_CELL_UPDATE = 21       # FP32-pipe instructions
OPS_PER_WINDOW_UPDATE = 3
FLOP_PER_CELL_UPDATE = 34
FLOP_PER_WINDOW_UPDATE = 5
# DRAM bytes (read + write) per patch-solve launch of this workload, measured by ncu
# (dram__bytes_read.sum + dram__bytes_write.sum) on the three level launches of
# `--case profile`: the same grids, bands and tiling as the timed step (the window
# length does not change it); 5.21 MB, 1.38 MB and 0.86 MB read, nothing written.
PATCH_DRAM_BYTES_PER_LAUNCH = (5206528 + 1382144 + 861952) / 3
# DRAM bytes per DNS launch on the 8192^2 grid, ncu on `--case dns-full` (two launches),
# by kernel; a kernel without a capture reports no traffic
DNS_DRAM_BYTES_PER_LAUNCH = {
    # 32-row tiles: 537.2 MB read + 236.1 MB written (algorithmic: 805.3 MB)
    "k_dns_step<32>": (537227776 + 237750016 + 537195776 + 234513664) / 2,
    # persistent, tensor copies, 32-row tiles: 537.3 MB read + 235.2 MB written
    "k_dns_tma<32,1>": (537318656 + 236889344 + 537293824 + 233592832) / 2,
}
WORKLOAD = "three_level_cellular"


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f)
    except OSError:
        return {}


# the profiling recipe's stand-ins, used (and named as such) only when the measured
# peaks file is absent
FALLBACK_PEAKS = {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0}


def _peak(key):
    """(value, source) of a roofline denominator: the measured figure, else the fallback."""
    v = _peaks().get(key)
    if v:
        return float(v), "measured (MEASURED_PEAKS.json)"
    return FALLBACK_PEAKS[key], "fallback (no measured peaks file)"


def _clock_sampler(path):
    q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
    try:
        return subprocess.Popen(["nvidia-smi", f"--query-gpu={q}", "--format=csv,noheader,nounits",
                                 "-lms", "200", "-i", str(_local_rank())],
                                stdout=open(path, "w"), stderr=subprocess.DEVNULL)
    except OSError:
        return None


def _clock_summary(path):
    sm, mx, reasons = [], [], set()
    names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
    try:
        for line in open(path):
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1])); mx.append(float(f[2]))
            except ValueError:
                continue
            for n, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(n)
    except OSError:
        pass
    if not sm:
        return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
    loaded = [s for s in sm if s > 0.5 * max(sm)] or sm
    return {"sm_mhz": statistics.median(loaded), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
            "samples": len(sm)}


def _local_rank():
    return int(os.environ.get("LOCAL_RANK", "0"))


def _workload():
    import inputs
    return inputs.config_problem(WORKLOAD)


def _oracle_nodes(cores, N):
    return [((37 * k + 5) % N, (59 * k + 3) % N) for k in range(cores)]


def _oracle_sample(cores):
    """Time the oracle (as it stands) on a bounded sample of the workload: the
    full Algorithm 3 chain (all levels, full relaxation window) for `cores`
    macro nodes.  Returns (cell-updates/s, seconds, description, nodes, K)."""
    import oracle
    cfg = _workload()
    N = cfg["n_macro"]
    nodes = _oracle_nodes(cores, N)
    t0 = time.perf_counter()
    K, steps = oracle.chain(cfg["spectrum"], cfg["edges"], cfg["patch_n"], N, cfg["kappa"], nodes,
                            cfl=cfg["cfl"], t_burn=8.0, t_avg=4.0, want_steps=True)
    dt = time.perf_counter() - t0
    n2 = np.array([n * n for n in cfg["patch_n"]], dtype=np.float64)
    cu = float(np.sum(2.0 * steps * n2[None, :]))
    sample = (f"{len(nodes)} of the {N * N} macro nodes: full 3-level chain of 64^2 patch "
              f"solves with the full 8+4 tau window")
    return cu / dt, dt, sample, nodes, K


def ranks_max(x, world, device):
    """Max of a per-rank float over the job (all_reduce MAX; the value itself at
    world 1).  Replicas share no data: this timing reduction is the only exchange."""
    if world <= 1:
        return float(x)
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_rate(units_per_rank, ms_max, world):
    """Whole-job throughput of `world` replicas: all units over the slowest rank's time."""
    return world * units_per_rank / (ms_max * 1e-3)


def _config(world):
    """The workload's config object, shared by both arms' JSON lines."""
    cfg = _workload()
    N = cfg["n_macro"]
    return {"workload": WORKLOAD, "n_macro": N, "patch_n": cfg["patch_n"][0],
            "levels": len(cfg["patch_n"]), "patches_per_level": N * N, "kappa": cfg["kappa"],
            "window": "8 tau burn-in + 4 tau average", "macro_T": cfg["T"],
            "l2": "flushed between steps (512 MiB write)",
            "parallelism": f"replicas x{world}" if world > 1 else "single GPU"}


def reference_arm(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    import oracle
    cores = oracle.num_threads()
    for _ in range(args.warmup):
        _oracle_sample(cores)
    vals, secs = [], []
    for _ in range(args.steps):
        v, dt, sample, _, _ = _oracle_sample(cores)
        vals.append(v); secs.append(dt)
    value = statistics.mean(vals)
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT,
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1e3 * statistics.mean(secs), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": _config(args.gpus),
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                         "sample": sample},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


DNS_BYTES_PER_CELL_STEP = 12     # read u, read psi, write u (both RK stages fused)


SUR_OCTAVES = ((16, 32, 64), (32, 64, 32), (64, 128, 32))   # (lo, hi, patch n) of each level
# the 4th octave at 128^2 (features on the 64^2 sub-lattice): its plain solve costs ~10 ms a
# patch, so it trains on 2 base sets of a 64 x 64 macro grid and tests on a 32 x 32 one
SUR_OCTAVE_128 = (8, 16, 128, 64, 2, 32)                      # (lo, hi, n, N train, bases, N test)
SUR_TRAIN_FLOW, SUR_TEST_FLOW = 1510004510, 20261204           # continuous-spectrum seeds


def _octave_level(seed, lo, hi, n, N, kappa):
    """One octave band (lo <= |k1|, |k2| < hi) of a continuous-spectrum realization as
    a one-level problem: patch side 2 pi / lo, n x n patches on an N x N macro grid."""
    from inputs import flows
    import paper_1510_00451_gb300 as mlsd
    full = flows.continuous_spectrum(256, seed=seed)
    a, b = np.abs(full.k1), np.abs(full.k2)
    keep = (a >= lo) & (a < hi) & (b >= lo) & (b < hi)
    band = flows.Spectrum(full.k1[keep], full.k2[keep], full.re[keep], full.im[keep])
    return mlsd.Levels(band, kappa, N, [float(lo), float(hi)], [n], patch_div=[lo], cfl=0.2)


def surrogate_case(N=256, epochs=400, members=4, hidden=256, batch=2048, lr=3e-3,
                   thresholds=(5e-4, 1e-3, 2e-3), seed=1510, large=False, bases=(1, 1, 1)):
    """Surrogate vs plain on three octave levels of the continuous-spectrum flow
    (kappa = 1e-3, N x N patches per level, full relaxation window): the 5th
    octave (16 <= |k| < 32, 64^2 patches), the 6th and the 7th (32^2).  Training
    data: one seeded base set on every patch of each level of one flow
    realization (3 N^2 plain solves); test: the same levels of ANOTHER
    realization (no patch psi seen in training) with a fresh base set.  Reports,
    per level and threshold, the fallback fraction, the K error against the plain
    solve and the K-tensor rate of both paths, and the totals over the levels.
    With large, the 4th octave at 128^2 patches joins (SUR_OCTAVE_128) and is
    reported on its own (not in the totals)."""
    import torch
    import inputs
    import paper_1510_00451_gb300 as mlsd
    from paper_1510_00451_gb300 import surrogate as S
    dev = torch.device("cuda", _local_rank())
    kappa = 1e-3
    P = N * N
    octs = [(lo, hi, n, N, nb, N) for (lo, hi, n), nb in zip(SUR_OCTAVES, bases)]
    if large:
        octs = octs + [SUR_OCTAVE_128]
    t0 = time.perf_counter()
    Xs, Ys = [], []
    for i, (lo, hi, n, Ntr, nb, _) in enumerate(octs):
        lv = _octave_level(SUR_TRAIN_FLOW, lo, hi, n, Ntr, kappa)
        base_sets = [inputs.random_bases(Ntr * Ntr, kappa, seed + 100 + i + 10 * j)
                     for j in range(nb)]
        X, Y = S.make_dataset(lv, 1, base_sets)
        Xs.append(X); Ys.append(Y)
        lv.close()
    X, Y = torch.cat(Xs), torch.cat(Ys)
    del Xs, Ys
    torch.cuda.synchronize()
    t_data = time.perf_counter() - t0
    sur = mlsd.Surrogate(members=members, hidden=hidden, max_batch=batch)
    for m in range(members):
        sur.set_params(m, inputs.mlp_init(mlsd.SUR_IN, hidden, seed * 10 + m))
    t0 = time.perf_counter()
    losses = sur.train(X, Y, epochs, batch, lr, lr_final=1e-5, seed=seed)
    torch.cuda.synchronize()
    t_train = time.perf_counter() - t0
    del X, Y
    stream = torch.cuda.current_stream()
    e0 = torch.cuda.Event(enable_timing=True); e1 = torch.cuda.Event(enable_timing=True)

    def timed(fn):
        e0.record(stream); r = fn(); e1.record(stream)
        torch.cuda.synchronize()
        return r, e0.elapsed_time(e1) * 1e-3

    levels, tot_plain, tot_sur, errs = [], 0.0, {t: 0.0 for t in thresholds}, {t: [] for t in thresholds}
    for i, (lo, hi, n, _, _, Nte) in enumerate(octs):
        P = Nte * Nte
        lv = _octave_level(SUR_TEST_FLOW, lo, hi, n, Nte, kappa)
        Bt = torch.tensor(inputs.random_bases(P, kappa, seed + 99 + i), dtype=torch.float64,
                          device=dev)
        Kp = torch.empty_like(Bt); Ks = torch.empty_like(Bt)
        if n <= 64:
            lv.solve_level(1, Bt, Kp)                   # warm-up
        _, t_plain = timed(lambda: lv.solve_level(1, Bt, Kp))
        Kpn = Kp.cpu().numpy()
        ok = np.isfinite(Kpn).all(1)                    # a non-finite plain solve has no reference
        rows = []
        in_total = n <= 64
        lv.solve_level_surrogate(sur, 1, Bt, Ks, 1e30)      # warm-up; the ensemble alone
        err0 = S.k_error(Ks.cpu().numpy()[ok], Kpn[ok])
        for thr in thresholds:
            nfb, t_sur = timed(lambda: lv.solve_level_surrogate(sur, 1, Bt, Ks, thr))
            err = S.k_error(Ks.cpu().numpy()[ok], Kpn[ok])
            if in_total:
                errs[thr].append(err)
                tot_sur[thr] += t_sur
            rows.append({"threshold": thr, "fallback_frac": nfb / P, "seconds": t_sur,
                         "k_tensors_per_s": P / t_sur, "speedup_vs_plain": t_plain / t_sur,
                         "k_rel_err": {"max": float(err.max()), "p99": float(np.quantile(err, 0.99)),
                                       "median": float(np.median(err)),
                                       "frac_le_1e-3": float(np.mean(err <= 1e-3))}})
        if in_total:
            tot_plain += t_plain
        levels.append({"octave": f"{lo}<=|k|<{hi}", "patch_n": n, "patches": P,
                       "plain_nonfinite": int((~ok).sum()),
                       "in_totals": in_total, "plain_seconds": t_plain,
                       "plain_k_tensors_per_s": P / t_plain,
                       "plain_cell_updates_per_s": lv.level_work(1)[0] / t_plain,
                       "ensemble_only": {"median": float(np.median(err0)),
                                         "frac_le_1e-3": float(np.mean(err0 <= 1e-3))},
                       "by_threshold": rows})
        assert lv.status() in (0, -5)                   # MLSD_ENONFINITE: counted above
        lv.close()
    overall = []
    P = N * N
    for thr in thresholds:
        err = np.concatenate(errs[thr])
        overall.append({"threshold": thr, "speedup_vs_plain": tot_plain / tot_sur[thr],
                        "k_tensors_per_s": len(SUR_OCTAVES) * P / tot_sur[thr],
                        "k_rel_err": {"max": float(err.max()), "p99": float(np.quantile(err, 0.99)),
                                      "median": float(np.median(err)),
                                      "frac_le_1e-3": float(np.mean(err <= 1e-3))}})
    # the tensor-core ensemble kernel alone on one level's rows
    Xt = torch.empty(P, mlsd.SUR_IN, dtype=torch.bfloat16, device=dev)
    lv = _octave_level(SUR_TEST_FLOW, 32, 64, 32, N, kappa)
    lv.features(1, torch.tensor(inputs.random_bases(P, kappa, seed), dtype=torch.float64,
                                device=dev), Xt)
    lv.close()
    out = torch.empty(members, P, 3, dtype=torch.float32, device=dev)
    sur.predict(Xt, out)
    _, t_mlp = timed(lambda: sur.predict(Xt, out))
    mlp_flop = 2.0 * P * members * (mlsd.SUR_IN * hidden + 2 * hidden * hidden + hidden * 16)
    assert sur.status() == 0
    peak, src = _peak("bf16_tflops")
    extra = (f"; plus octave 8-16 at 128^2 ({SUR_OCTAVE_128[3] ** 2 * SUR_OCTAVE_128[4]} "
             f"training solves, {SUR_OCTAVE_128[5] ** 2} test patches, outside the totals)"
             if large else "")
    return {"workload": f"continuous-spectrum octaves 16-32 (64^2), 32-64, 64-128 (32^2), {P} "
                        "patches each, kappa=1e-3, full window; trained on one flow "
                        f"realization ({sum(bases) * P} plain solves, {list(bases)} base sets "
                        "per level), tested on another"
                        + extra,
            "members": members, "hidden": hidden, "epochs": epochs, "batch": batch,
            "final_loss": losses, "levels": levels, "overall": overall,
            "plain_k_tensors_per_s": len(SUR_OCTAVES) * P / tot_plain,
            "mlp_tensor_core": {"ms": t_mlp * 1e3, "achieved_tflops": mlp_flop / t_mlp / 1e12,
                                "peak_bf16_tflops": peak, "peak_source": src,
                                "frac": mlp_flop / t_mlp / 1e12 / peak,
                                "bound": "tensor", "unit": "TFLOP/s",
                                "kernel": "k_mlp_tma (k_mlp_tc where tensor maps are unavailable)"},
            "seconds": {"dataset": t_data, "train": t_train, "plain": tot_plain}}


def _profile_gap(a, b):
    """max |a - b| and relative L2 of two x1-profiles."""
    a = np.asarray(a, dtype=np.float64); b = np.asarray(b, dtype=np.float64)
    return {"max_abs": float(np.abs(a - b).max()),
            "rel_l2": float(np.linalg.norm(a - b) / np.linalg.norm(b))}


def _fit_k11(profile, t_end, u_left=1.0, u_right=0.0):
    """K11 of the constant-K homogenized problem whose x1-profile at t_end best
    fits `profile` (values at x1 = 2 pi i / n, i = 0..n-1; Dirichlet at x1 = 0 and
    2 pi, step start): the semi-discrete solution on the same n columns is
    l_i + sum_p c_p exp(-K11 lambda_p t) sin(pi p i / n), l the linear profile,
    lambda_p = 4 sin^2(pi p / 2n) / H^2, c_p the sine coefficients of the step
    minus l.  Golden-section search on log K11."""
    import inputs
    n = len(profile)
    H = 2 * math.pi / n
    i = np.arange(n)
    lin = u_left + (u_right - u_left) * i / n
    u0 = inputs.step_u0(n, u_left, u_right)[0]
    p = np.arange(1, n)
    S = np.sin(np.pi * np.outer(p, i) / n)                     # [p][i]
    c = (2.0 / n) * S @ (u0 - lin)
    lam = 4 * np.sin(np.pi * p / (2 * n)) ** 2 / H ** 2

    def gap(lk):
        return float(np.linalg.norm(lin + (c * np.exp(-math.exp(lk) * lam * t_end)) @ S - profile))
    lo, hi = math.log(1e-3), math.log(1e3)
    for _ in range(80):
        a1 = hi - 0.618 * (hi - lo); a2 = lo + 0.618 * (hi - lo)
        if gap(a1) < gap(a2):
            hi = a2
        else:
            lo = a1
    return math.exp(0.5 * (lo + hi))


def _sec4_compare(spec, edges, patch_n, patch_div, N, nf, t_end, kappa=1.0):
    """SHMM (level chain with the full relaxation window, macro solve on N x N)
    against the direct simulation on nf x nf, both with the Sec. 4 boundaries,
    from the step; x2-averaged profiles and the K11 fitted to the DNS profile."""
    import torch
    import inputs
    import paper_1510_00451_gb300 as mlsd
    dev = torch.device("cuda", _local_rank())
    r = nf // N
    t0 = time.perf_counter()
    lv = mlsd.Levels(spec, kappa, N, edges, patch_n, patch_div=patch_div, cfl=0.2)
    K = torch.zeros(N * N, 3, dtype=torch.float64, device=dev)
    lv.effective_diffusivity(K)
    torch.cuda.synchronize()
    t_chain = time.perf_counter() - t0
    assert lv.status() == 0
    sizes = [sorted(set(int(x) for x in lv.patch_sizes(l + 1))) for l in range(len(edges) - 1)]
    lv.close()

    def macro(Kf):
        dt = mlsd.macro_dt(Kf, N, 0.2)
        ns = max(1, math.ceil(t_end / dt))
        U = torch.tensor(inputs.step_u0(N), dtype=torch.float64, device=dev)
        mlsd.macro_step_dirichlet(U, Kf, t_end / ns, ns, 1.0, 0.0)
        return U.cpu().numpy().mean(0)

    def dns(psi):
        # FP64: ~5e5 steps of a relaxing profile stall in FP32 (increments below half an ulp)
        dt = mlsd.dns_dt(psi, kappa, 0.2)
        ns = math.ceil(t_end / dt)
        u = torch.tensor(inputs.step_u0(nf), dtype=torch.float64, device=dev)
        ut = torch.empty_like(u)
        mlsd.dns_run_dirichlet(u, ut, psi, kappa, t_end / ns, ns, 1.0, 0.0)
        torch.cuda.synchronize()
        return u.cpu().numpy().mean(0), ns

    prof_shmm = macro(K)
    prof_none = macro(torch.tensor(np.tile([kappa, 0.0, kappa], (N * N, 1)), dtype=torch.float64,
                                   device=dev))
    psi = torch.empty(nf, nf, dtype=torch.float32, device=dev)
    mlsd.grid_psi(spec, nf, psi)
    t0 = time.perf_counter()
    prof_dns, ns = dns(psi)
    t_dns = time.perf_counter() - t0
    Kn = K.cpu().numpy()
    return {"K_shmm_mean": Kn.mean(0).tolist(), "K_shmm_min": Kn.min(0).tolist(),
            "K_shmm_max": Kn.max(0).tolist(), "patch_sizes": sizes,
            "K11_dns_fit": _fit_k11(prof_dns, t_end),
            "K11_shmm_profile_fit": _fit_k11(prof_shmm, t_end),
            "shmm_vs_dns": _profile_gap(prof_shmm, prof_dns[::r]),
            "no_advection_vs_dns": _profile_gap(prof_none, prof_dns[::r]),
            "dns": {"grid": nf, "steps": ns, "dt": t_end / ns, "seconds": t_dns},
            "chain_seconds": t_chain}


def sec4_case(N=64, nf=512, t_end=0.4 * math.pi ** 2):
    """The paper's Sec. 4 set-up (kappa = 1, u = 1 at x1 = 0 and 0 at x1 = 2 pi,
    periodic in x2, step initial condition, t_end = 0.4 pi^2: the paper's t = 0.1
    on [0,1]^2 under x -> 2 pi x, t -> 4 pi^2 t) on two of its flows:
    * two separated cellular modes (Sec. 4.2): psi = a (sin 5x sin 5y + sin 25x
      sin 25y), a = 1/3 (printed) and 2.5 (K near the printed values); two levels
      (edges 1, 6, 26; patch sides 2 pi and 2 pi / 5; 64^2 patches);
    * a continuous spectrum (Sec. 4.4): random phases, 1 <= |k| <= 50, |psi_hat|
      ~ |k|^-3, rms speed 4; three levels (edges 1, 5, 25, 51; patch sides 2 pi,
      2 pi / 5, 2 pi / 25; sizes by the size rule).
    SHMM: the full relaxation window, then the macro solve on N x N.  Reference:
    the direct simulation on nf x nf (the paper's 512^2), and the same without the
    flow (its fit checks the K11 fit, which should return kappa).  Compared: the
    x2-averaged profiles at the macro nodes and K11 fitted to each profile."""
    import torch
    import inputs
    from inputs import flows
    import paper_1510_00451_gb300 as mlsd
    dev = torch.device("cuda", _local_rank())
    zero = torch.zeros(nf, nf, dtype=torch.float32, device=dev)
    dt = mlsd.dns_dt(zero, 1.0, 0.2)
    ns = math.ceil(t_end / dt)
    u = torch.tensor(inputs.step_u0(nf), dtype=torch.float64, device=dev)
    mlsd.dns_run_dirichlet(u, torch.empty_like(u), zero, 1.0, t_end / ns, ns, 1.0, 0.0)
    k11_noflow = _fit_k11(u.cpu().numpy().mean(0), t_end)
    cases = []
    for amp in (1.0 / 3.0, 2.5):
        spec = flows.cellular([(amp, 5, 5), (amp, 25, 25)])
        r = _sec4_compare(spec, [1.0, 6.0, 26.0], [64, 64], [1, 5], N, nf, t_end)
        cases.append({"flow": f"two cellular modes (5, 25), a = {amp:.4g}", **r})
    # the continuous spectrum's K is larger: at t_end its profile is nearly relaxed,
    # so it is compared at t_end / 4 (the paper's t = 0.025)
    spec = flows.continuous_spectrum(50, seed=1510004510, slope=-3.0, vrms=4.0)
    r = _sec4_compare(spec, [1.0, 5.0, 25.0, 51.0], [0, 0, 0], [1, 5, 25], N, nf, t_end / 4)
    cases.append({"flow": "continuous spectrum 1 <= |k| <= 50, |psi_hat| ~ k^-3, rms speed 4",
                  "t": t_end / 4, **r})
    return {"workload": f"Sec. 4 set-up: kappa=1, Dirichlet x1 / periodic x2, step IC, "
                        f"t={t_end:.4f}; SHMM on {N}^2 macro nodes; DNS {nf}^2",
            "K11_fit_of_the_no_flow_dns": k11_noflow, "cases": cases}


def _fit_k_periodic(U0, U, t_end):
    """Constant K (K11, K12, K22) of the periodic homogenized problem whose
    solution from U0 best fits U at t_end on the N x N macro grid: each Fourier
    mode decays as exp(-t lambda), lambda = [4 K11 sin^2(t1/2) + 4 K22 sin^2(t2/2)
    + 2 K12 sin t1 sin t2] / H^2 (the macro scheme's semi-discrete symbol)."""
    from scipy.optimize import least_squares
    N = U0.shape[0]
    H = 2 * math.pi / N
    th = 2 * math.pi * np.fft.fftfreq(N)
    t1, t2 = th[None, :], th[:, None]
    F0, F1 = np.fft.fft2(U0), np.fft.fft2(U)

    def res(q):
        k11, k22, c = math.exp(q[0]), math.exp(q[1]), math.tanh(q[2])
        k12 = c * math.sqrt(k11 * k22)
        lam = (4 * k11 * np.sin(t1 / 2) ** 2 + 4 * k22 * np.sin(t2 / 2) ** 2
               + 2 * k12 * np.sin(t1) * np.sin(t2)) / H ** 2
        d = F0 * np.exp(-t_end * lam) - F1
        return np.concatenate([d.real.ravel(), d.imag.ravel()])
    q = least_squares(res, [0.0, 0.0, 0.0]).x
    k11, k22 = math.exp(q[0]), math.exp(q[1])
    return [k11, math.tanh(q[2]) * math.sqrt(k11 * k22), k22]


def spectrum_dns_case(N=16, nf=8192, t_end=1.0):
    """The full SHMM pipeline on the continuous-spectrum flow (|k| <= 256,
    kappa = 1e-3, 8 octave levels, sizes by the size rule): the level chain with
    the full 8 tau + 4 tau relaxation window on the N x N macro grid, then the
    macro solve of the Gaussian (sigma = 0.5) to t_end, against the direct
    simulation on nf x nf to the same time coarse-grained onto the macro grid
    (the structure of the paper's Sec. 4.4 comparison).  Also the pure-diffusion
    macro solution, and the constant K fitted to each solution."""
    import torch
    import inputs
    import paper_1510_00451_gb300 as mlsd
    dev = torch.device("cuda", _local_rank())
    cfg = inputs.config_problem("continuous_spectrum")
    Lc = len(cfg["edges"]) - 1
    t0 = time.perf_counter()
    lv = mlsd.Levels(cfg["spectrum"], cfg["kappa"], N, cfg["edges"], [0] * Lc, cfl=cfg["cfl"])
    K = torch.zeros(N * N, 3, dtype=torch.float64, device=dev)
    lv.effective_diffusivity(K)
    torch.cuda.synchronize()
    t_chain = time.perf_counter() - t0
    assert lv.status() == 0
    work = sum(lv.level_work(l + 1)[0] for l in range(Lc))
    lv.close()
    U0 = inputs.gaussian_u0(N, cfg["sigma"])

    def macro(Kf):
        dt = mlsd.macro_dt(Kf, N, cfg["cfl"])
        ns = max(1, math.ceil(t_end / dt))
        U = torch.tensor(U0, dtype=torch.float64, device=dev)
        mlsd.macro_step(U, Kf, t_end / ns, ns, want_mass=False)
        return U.cpu().numpy()

    U_shmm = macro(K)
    U_none = macro(torch.tensor(np.tile([cfg["kappa"], 0.0, cfg["kappa"]], (N * N, 1)),
                                dtype=torch.float64, device=dev))
    psi = torch.empty(nf, nf, dtype=torch.float32, device=dev)
    mlsd.grid_psi(cfg["spectrum"], nf, psi)
    dt = mlsd.dns_dt(psi, cfg["kappa"], cfg["cfl"])
    ns = math.ceil(t_end / dt)
    u = torch.tensor(inputs.gaussian_u0(nf, cfg["sigma"]), dtype=torch.float32, device=dev)
    ut = torch.empty_like(u)
    t0 = time.perf_counter()
    mlsd.dns_run(u, ut, psi, cfg["kappa"], t_end / ns, ns)
    torch.cuda.synchronize()
    t_dns = time.perf_counter() - t0
    Ud = torch.empty(N, N, dtype=torch.float32, device=dev)
    mlsd.coarse_grain(u, N, Ud)
    U_dns = Ud.cpu().numpy().astype(np.float64)
    # coarse-grained initial field: the DNS's own start on the macro grid
    U0c = torch.empty(N, N, dtype=torch.float32, device=dev)
    mlsd.coarse_grain(torch.tensor(inputs.gaussian_u0(nf, cfg["sigma"]), dtype=torch.float32,
                                   device=dev), N, U0c)
    U0c = U0c.cpu().numpy().astype(np.float64)

    def dev_gap(a, b):
        a = a - a.mean(); b = b - b.mean()
        return float(np.linalg.norm(a - b) / np.linalg.norm(b))
    Kn = K.cpu().numpy()
    return {"workload": f"continuous spectrum |k|<=256, kappa=1e-3, 8 levels, {N}^2 macro "
                        f"nodes, full window; Gaussian sigma=0.5 to t={t_end}; DNS {nf}^2",
            "K_shmm_mean": Kn.mean(0).tolist(), "K_shmm_min": Kn.min(0).tolist(),
            "K_shmm_max": Kn.max(0).tolist(),
            "K_fit_dns": _fit_k_periodic(U0c, U_dns, t_end),
            "K_fit_shmm": _fit_k_periodic(U0, U_shmm, t_end),
            "shmm_vs_dns_rel_l2_of_deviation": dev_gap(U_shmm, U_dns),
            "no_advection_vs_dns_rel_l2_of_deviation": dev_gap(U_none, U_dns),
            "chain_seconds": t_chain, "chain_cell_updates": work,
            "dns": {"grid": nf, "steps": ns, "dt": t_end / ns, "seconds": t_dns}}


def offdiag_case(N=4):
    """The Sec. 4.3 stress test of the off-diagonal closed forms, at half the
    paper's wavenumbers (alpha = 2 instead of 5, so that the fully resolved
    reference fits one 256^2 patch): psi = a(phi_c(2,2) + phi_c(2,18) +
    phi_c(18,2) + phi_c(20,20)), phi_c(a,b) = sin(a x1) sin(b x2), kappa = 1,
    a = 1/5 (the printed amplitude) and 1.
    SHMM: two levels (edges 1, 3, 21; patch sides 2 pi and pi; the (2,18),
    (18,2) pair is level 1's psi_12, psi_21 and enters through Algorithms 1-2),
    full relaxation window, N x N macro nodes.  Reference: one patch of side
    2 pi with every mode in its band (256^2: 12.8 points per wavelength of
    mode 20).  Also both without the off-diagonal pair."""
    import torch
    from inputs import flows
    import paper_1510_00451_gb300 as mlsd
    dev = torch.device("cuda", _local_rank())

    def shmm(terms):
        lv = mlsd.Levels(flows.cellular(terms), 1.0, N, [1.0, 3.0, 21.0], [32, 128],
                         patch_div=[1, 2], cfl=0.2)
        K = torch.zeros(N * N, 3, dtype=torch.float64, device=dev)
        lv.effective_diffusivity(K)
        assert lv.status() == 0
        lv.close()
        Kn = K.cpu().numpy()
        return Kn.mean(0), float(np.abs(Kn - Kn.mean(0)).max())

    def full(terms):
        lv = mlsd.Levels(flows.cellular(terms), 1.0, 1, [1.0, 21.0], [256], patch_div=[1],
                         cfl=0.2)
        K = torch.zeros(1, 3, dtype=torch.float64, device=dev)
        B = torch.tensor([[1.0, 0.0, 1.0]], dtype=torch.float64, device=dev)
        lv.solve_level(1, B, K)
        assert lv.status() == 0
        lv.close()
        return K.cpu().numpy()[0]

    def rel(a, b):
        return float(np.linalg.norm(np.asarray(a) - b) / np.linalg.norm(b))
    t0 = time.perf_counter()
    cases = []
    for a in (0.2, 1.0):            # the printed amplitude 1/5, and a stronger flow
        diag = [(a, 2, 2), (a, 20, 20)]
        off = [(a, 2, 18), (a, 18, 2)]
        K_s, spread = shmm(diag + off)
        K_f = full(diag + off)
        K_s0, _ = shmm(diag)
        K_f0 = full(diag)
        cases.append({"amplitude": a, "K_shmm": K_s.tolist(), "K_shmm_node_spread": spread,
                      "K_full_patch": K_f.tolist(), "rel_err_shmm_vs_full": rel(K_s, K_f),
                      "without_offdiagonal_pair": {"K_shmm": K_s0.tolist(),
                                                   "K_full_patch": K_f0.tolist(),
                                                   "rel_err": rel(K_s0, K_f0)}})
    torch.cuda.synchronize()
    return {"workload": "Sec. 4.3 structure at alpha = 2: psi = a(phi_c(2,2) + phi_c(2,18) + "
                        "phi_c(18,2) + phi_c(20,20)), kappa = 1; SHMM 2 levels (32^2, 128^2 "
                        f"patches, {N}^2 nodes, full window) vs one fully resolved 256^2 patch",
            "cases": cases, "seconds": time.perf_counter() - t0}


def geometry_case(N=32):
    """Patch geometry and periodisation on the two-scale cellular flow
    (psi = sin x sin y + sin 8x sin 8y, kappa = 0.05, 2 levels, 32^2 patches,
    N x N macro nodes, full relaxation window, FP32): patches of one period of
    each level's band (the default), and the paper's local domains of side 2H
    (H = 2 pi / N) on which neither band is periodic, with the band wrapped at
    the seam or replaced by its periodic component (periodic-plus-smooth)."""
    import torch
    from inputs import flows
    import paper_1510_00451_gb300 as mlsd
    dev = torch.device("cuda", _local_rank())
    spec = flows.cellular_two_scale(1.0, 1.0, 8)
    out = []
    for name, div, per in (("one period of each band", None, False),
                           ("side 2H, band wrapped at the seam", [N // 2, N // 2], False),
                           ("side 2H, periodic component of the band", [N // 2, N // 2], True)):
        lv = mlsd.Levels(spec, 0.05, N, [1.0, 8.0, 9.0], [32, 32], patch_div=div, periodize=per,
                         cfl=0.2)
        K = torch.zeros(N * N, 3, dtype=torch.float64, device=dev)
        lv.effective_diffusivity(K)
        rc = lv.status()
        steps = [lv.level_work(l + 1)[1] for l in range(2)]
        lv.close()
        Kn = K.cpu().numpy()
        out.append({"geometry": name, "status": mlsd.ERRORS.get(rc, rc),
                    "max_steps_per_level": steps, "K_mean": Kn.mean(0).tolist(),
                    "K_min": Kn.min(0).tolist(), "K_max": Kn.max(0).tolist()})
    return {"workload": f"two-scale cellular flow, kappa=0.05, {N}^2 macro nodes, 32^2 patches, "
                        "full window, FP32", "variants": out}


def uneven_case(n_avg=256):
    """The continuous-spectrum workload at full size: |k| <= 256, 8 octave levels,
    256 x 256 macro nodes (65536 patches per level), patch sizes 32^2 .. 256^2
    from the size rule, every level's size classes launched concurrently inside
    one captured graph.  Fixed n_avg-step window per patch (the full window of
    the 256^2 levels needs ~5e5 steps).  Also per level and per patch size: the
    patch kernels' device time (CUDA events around each launch, in a second pass
    outside the graph with the sizes of a level run one after another) and its
    cell-update rate and FP32-issue fraction."""
    import torch
    import inputs
    import paper_1510_00451_gb300 as mlsd
    cfg = inputs.config_problem("continuous_spectrum")
    N, L = cfg["n_macro"], len(cfg["edges"]) - 1
    t0 = time.perf_counter()
    lv = mlsd.Levels(cfg["spectrum"], cfg["kappa"], N, cfg["edges"], [0] * L, cfl=cfg["cfl"],
                     n_burn_fixed=0, n_avg_fixed=n_avg)
    t_setup = time.perf_counter() - t0
    hist = []
    for l in range(1, L + 1):
        sz = lv.patch_sizes(l)
        vals, cnt = np.unique(sz, return_counts=True)
        hist.append({int(v): int(c) for v, c in zip(vals, cnt)})
    dev = torch.device("cuda", _local_rank())
    K = torch.zeros(N * N, 3, dtype=torch.float64, device=dev)
    lv.effective_diffusivity(K)                   # capture + warm-up
    torch.cuda.synchronize()
    stream = torch.cuda.current_stream()
    e0 = torch.cuda.Event(enable_timing=True); e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream); lv.effective_diffusivity(K); e1.record(stream)
    torch.cuda.synchronize()
    t = e0.elapsed_time(e1) * 1e-3
    assert lv.status() == 0
    work = [lv.level_work(l + 1) for l in range(L)]
    cu = sum(w[0] for w in work)
    # per level and per patch size: a second pass outside the graph with each level's
    # size classes run one after another (profiling mode 2), so that every class's
    # events time it alone; the chain above runs them concurrently
    for l in range(L):
        lv.profile_collect(l + 1)
    lv.profile(True, serial_classes=True)
    lv.effective_diffusivity(K)
    torch.cuda.synchronize()
    lv.profile(False)
    peaks = _peaks()
    sm_count = torch.cuda.get_device_properties(dev).multi_processor_count
    issue_peak = sm_count * 128 * peaks.get("sm_max_mhz", 2070.0) * 1e6
    per_level = []
    for l in range(L):
        cls = lv.profile_collect_classes(l + 1)
        ms = sum(v[0] for v in cls.values())
        n = sum(v[1] for v in cls.values())
        cu_l, _, wu_l = work[l]
        ops = cu_l * OPS_PER_CELL_UPDATE + wu_l * OPS_PER_WINDOW_UPDATE
        classes = []
        for size, (ms_c, n_c) in sorted(cls.items()):
            if size == 0 or ms_c <= 0:
                continue
            # fixed window without burn-in: every step of every field is inside it
            cu_c = hist[l][size] * 2 * size * size * n_avg
            classes.append({"n": size, "patches": hist[l][size], "kernel_ms": ms_c,
                            "cell_updates_per_s": cu_c / (ms_c * 1e-3),
                            "fp32_issue_frac": cu_c * (OPS_PER_CELL_UPDATE + OPS_PER_WINDOW_UPDATE)
                                               / (ms_c * 1e-3) / issue_peak})
        per_level.append({"level": l + 1, "sizes": hist[l], "kernel_ms": ms, "launches": n,
                          "cell_updates": cu_l,
                          "cell_updates_per_s": cu_l / (ms * 1e-3) if ms > 0 else None,
                          "fp32_issue_frac": ops / (ms * 1e-3) / issue_peak if ms > 0 else None,
                          "classes": classes})
    tiles = [lv.info(l + 1) for l in range(L)]
    ops = sum(w[0] * OPS_PER_CELL_UPDATE + w[2] * OPS_PER_WINDOW_UPDATE for w in work)
    return {"workload": "continuous spectrum |k|<=256, 8 octave levels, 65536 patches/level, "
                        f"sizes 32^2..256^2 by the size rule, {n_avg}-step window",
            "cell_updates_per_s": cu / t, "seconds": t, "cell_updates": cu,
            "fp32_issue_frac": ops / t / issue_peak,
            "k_eff_tensors_per_s": N * N / t, "setup_s": t_setup,
            "per_level": per_level,
            "largest_class_tiling": [f"{i['tile_bx']}x{i['tile_by']} c{i['cluster']} m{i['min_ctas']}"
                                     f"{' packed' if i['packed'] else ''}"
                                     f"{' sync%d' % i['split'] if i['split'] else ''}"
                                     f"{' tmem' if i['coef_tmem'] == 1 else ''}"
                                     f"{' tmem-lazy' if i['coef_tmem'] == 2 else ''}"
                                     f" n={i['n']}" for i in tiles],
            "level_launch": ["one launch" if i["level_launch"] else
                             ("per-size launches" if i["n_classes"] > 1 else "one size")
                             for i in tiles],
            "finite": bool(torch.isfinite(K).all().item())}


def cluster_case(N=32, n_burn=32, n_avg=32):
    """The first octave level of the continuous-spectrum flow with 256^2 patches
    (each field split over a thread-block cluster) on an N x N macro grid, fixed
    window: the launch shape of the largest size class, small enough to profile."""
    import torch
    import inputs
    import paper_1510_00451_gb300 as mlsd
    cfg = inputs.config_problem("continuous_spectrum")
    lv = mlsd.Levels(cfg["spectrum"], cfg["kappa"], N, cfg["edges"][:2], [256], cfl=cfg["cfl"],
                     n_burn_fixed=n_burn, n_avg_fixed=n_avg)
    K = torch.zeros(N * N, 3, dtype=torch.float64, device=torch.device("cuda", _local_rank()))
    lv.effective_diffusivity(K)
    torch.cuda.synchronize()
    stream = torch.cuda.current_stream()
    e0 = torch.cuda.Event(enable_timing=True); e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream); lv.effective_diffusivity(K); e1.record(stream)
    torch.cuda.synchronize()
    t = e0.elapsed_time(e1) * 1e-3
    rc = lv.status()
    cu = lv.level_work(1)[0]
    i = lv.info(1)
    print(json.dumps({"case": "cluster-profile", "status": rc, "cell_updates_per_s": cu / t,
                      "seconds": t, "tiling": f"{i['tile_bx']}x{i['tile_by']} c{i['cluster']} "
                      f"m{i['min_ctas']}{' sync%d' % i['split'] if i['split'] else ''}"
                      f"{' tmem' if i['coef_tmem'] == 1 else ''}{' tmem-lazy' if i['coef_tmem'] == 2 else ''}",
                      "finite": bool(torch.isfinite(K).all().item())}), flush=True)
    return 0 if rc == 0 else 1


def mlp_case(M=65536, members=4, hidden=256):
    """One tensor-core ensemble inference on M random feature rows (ncu case)."""
    import torch
    import inputs
    import paper_1510_00451_gb300 as mlsd
    dev = torch.device("cuda", _local_rank())
    sur = mlsd.Surrogate(members=members, hidden=hidden, max_batch=1024)
    for m in range(members):
        sur.set_params(m, inputs.mlp_init(mlsd.SUR_IN, hidden, m))
    g = torch.Generator(device=dev); g.manual_seed(0)
    X = torch.randn(M, mlsd.SUR_IN, device=dev, generator=g).to(torch.bfloat16)
    out = torch.empty(members, M, 3, device=dev)
    sur.predict(X, out)
    sur.predict(X, out)
    stream = torch.cuda.current_stream()
    e0 = torch.cuda.Event(enable_timing=True); e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(5):
        sur.predict(X, out)
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / 5
    flop = 2.0 * M * members * (mlsd.SUR_IN * hidden + 2 * hidden * hidden + hidden * 16)
    ok = sur.status() == 0 and bool(torch.isfinite(out).all().item())
    print(json.dumps({"case": "mlp-profile", "ok": ok, "rows": M, "ms": ms,
                      "tflops": flop / (ms * 1e-3) / 1e12}), flush=True)
    return 0 if ok else 1


def series_case(N=256, reps=3):
    """Surrogate features of every patch of the 6th-octave level (65536 patches of
    32^2): k_features (DFT window) and k_series (moments T_2..T_19 by FFTs and
    their resummation), timed with CUDA events (ncu case)."""
    import torch
    import inputs
    import paper_1510_00451_gb300 as mlsd
    dev = torch.device("cuda", _local_rank())
    lv = _octave_level(SUR_TEST_FLOW, 32, 64, 32, N, 1e-3)
    P = N * N
    B = torch.tensor(inputs.random_bases(P, 1e-3, 3), dtype=torch.float64, device=dev)
    X = torch.empty(P, mlsd.SUR_IN, dtype=torch.bfloat16, device=dev)
    lv.features(1, B, X)
    stream = torch.cuda.current_stream()
    e0 = torch.cuda.Event(enable_timing=True); e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(reps):
        lv.features(1, B, X)
    e1.record(stream)
    torch.cuda.synchronize()
    ok = lv.status() == 0 and bool(torch.isfinite(X.float()).all().item())
    print(json.dumps({"case": "series-profile", "ok": ok, "patches": P,
                      "ms_per_call": e0.elapsed_time(e1) / reps}), flush=True)
    return 0 if ok else 1


def train_case(rows=16384, epochs=2, members=4, hidden=256, batch=2048):
    """Surrogate training steps on random rows of the training shape (ncu case):
    `epochs` passes of rows / batch Adam steps per member, timed with CUDA events
    after one untimed epoch."""
    import torch
    import inputs
    import paper_1510_00451_gb300 as mlsd
    dev = torch.device("cuda", _local_rank())
    sur = mlsd.Surrogate(members=members, hidden=hidden, max_batch=batch)
    for m in range(members):
        sur.set_params(m, inputs.mlp_init(mlsd.SUR_IN, hidden, m))
    g = torch.Generator(device=dev); g.manual_seed(0)
    X = (0.5 * torch.randn(rows, mlsd.SUR_IN, device=dev, generator=g)).to(torch.bfloat16)
    Y = 0.1 * torch.randn(rows, 3, device=dev, generator=g)
    sur.train(X, Y, 1, batch, 3e-3)
    stream = torch.cuda.current_stream()
    e0 = torch.cuda.Event(enable_timing=True); e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    losses = sur.train(X, Y, epochs, batch, 3e-3, lr_final=1e-3, seed=1)
    e1.record(stream)
    torch.cuda.synchronize()
    steps = members * epochs * (rows // batch)
    ms = e0.elapsed_time(e1) / steps
    # forward and weight gradients of the 4 layers, data gradients of layers 2..4
    per_row = 2 * (mlsd.SUR_IN * hidden + 2 * hidden * hidden + hidden * 3)
    flop = batch * (2 * per_row + 2 * (2 * hidden * hidden + hidden * 3))
    ok = sur.status() == 0 and all(math.isfinite(x) for x in losses)
    print(json.dumps({"case": "train-profile", "ok": ok, "steps": steps, "ms_per_step": ms,
                      "gflop_per_step": flop / 1e9, "tflops": flop / (ms * 1e-3) / 1e12}),
          flush=True)
    return 0 if ok else 1


def dns_case(nf, steps, warmup=20, report=False):
    """Direct simulation of the continuous-spectrum flow (|k| <= 256, kappa = 1e-3)
    on an nf x nf FP32 grid: `steps` fused RK2 steps timed with CUDA events."""
    import torch
    import inputs
    import paper_1510_00451_gb300 as mlsd
    dev = torch.device("cuda", _local_rank())
    cfg = inputs.config_problem("continuous_spectrum")
    psi = torch.empty(nf, nf, dtype=torch.float32, device=dev)
    mlsd.grid_psi(cfg["spectrum"], nf, psi)
    dt = mlsd.dns_dt(psi, cfg["kappa"], cfg["cfl"])
    u0 = torch.tensor(inputs.gaussian_u0(nf, cfg["sigma"]), dtype=torch.float32, device=dev)
    u = u0.clone()
    ut = torch.empty_like(u)
    mlsd.dns_run(u, ut, psi, cfg["kappa"], dt, warmup)
    u.copy_(u0)
    stream = torch.cuda.current_stream()
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True); e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    mlsd.dns_run(u, ut, psi, cfg["kappa"], dt, steps)
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    N = cfg["n_macro"]
    U = torch.empty(N, N, dtype=torch.float32, device=dev)
    mass = mlsd.coarse_grain(u, N, U)
    m0 = mlsd.coarse_grain(u0, N, U.clone())
    out = {"grid": nf, "steps": steps, "dt": dt, "ms": ms, "kernel": mlsd.dns_kernel(),
           "cell_steps_per_s": nf * nf * steps / (ms * 1e-3),
           "mass_rel_drift": abs(mass - m0) / m0,
           "finite": bool(torch.isfinite(u).all().item())}
    if report:
        print(json.dumps({"case": "dns-profile", **out}), flush=True)
        return 0 if out["finite"] else 1
    return out


def profile_case():
    """The benchmark's levels and launch shapes with a 200-step window per patch."""
    import torch
    import paper_1510_00451_gb300 as mlsd
    cfg = _workload()
    N = cfg["n_macro"]
    lv = mlsd.Levels(cfg["spectrum"], cfg["kappa"], N, cfg["edges"], cfg["patch_n"],
                     cfl=cfg["cfl"], n_burn_fixed=100, n_avg_fixed=100, precision=cfg["precision"])
    K = torch.zeros(N * N, 3, dtype=torch.float64, device="cuda:0")
    lv.effective_diffusivity(K)
    torch.cuda.synchronize()
    stream = torch.cuda.current_stream()
    e0 = torch.cuda.Event(enable_timing=True); e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream); lv.effective_diffusivity(K); e1.record(stream)
    torch.cuda.synchronize()
    rc = lv.status()
    work = sum(lv.level_work(l + 1)[0] for l in range(len(cfg["patch_n"])))
    i = lv.info(1)
    print(json.dumps({"case": "profile", "status": rc, "cell_updates": work,
                      "cell_updates_per_s": work / (e0.elapsed_time(e1) * 1e-3),
                      "tiling": f"{i['tile_bx']}x{i['tile_by']} m{i['min_ctas']}"
                                f"{' packed' if i['packed'] else ''}{' split' if i['split'] else ''}",
                      "K0": K[0].tolist()}), flush=True)
    return 0 if rc == 0 else 1


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=2)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="mlsd", choices=["mlsd", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-dns", action="store_true")
    ap.add_argument("--no-surrogate", action="store_true")
    ap.add_argument("--no-uneven", action="store_true")
    ap.add_argument("--no-experiments", action="store_true",
                    help="skip the Sec. 4 comparisons (set-up, off-diagonal stress, geometry)")
    ap.add_argument("--case", default="full",
                    choices=["full", "profile", "dns-profile", "dns-full", "surrogate",
                             "surrogate-large", "uneven",
                             "mlp-profile", "cluster-profile", "train-profile", "sec4",
                             "spectrum-dns", "offdiag", "geometry", "series-profile"],
                    help="profile: one pass of the same workload with a fixed 200-step window "
                         "per patch (a small case for ncu captures); prints no bench line")
    args = ap.parse_args()
    if args.impl == "reference":
        return reference_arm(args)
    if args.case == "profile":
        return profile_case()
    if args.case == "dns-profile":
        return dns_case(4096, 20, warmup=2, report=True)
    if args.case == "dns-full":
        return dns_case(8192, 10, warmup=2, report=True)
    if args.case == "surrogate":
        print(json.dumps({"case": "surrogate", **surrogate_case()}), flush=True)
        return 0
    if args.case == "surrogate-large":
        print(json.dumps({"case": "surrogate-large", **surrogate_case(large=True)}), flush=True)
        return 0
    if args.case == "mlp-profile":
        return mlp_case()
    if args.case == "cluster-profile":
        return cluster_case()
    if args.case == "train-profile":
        return train_case()
    if args.case == "uneven":
        print(json.dumps({"case": "uneven", **uneven_case()}), flush=True)
        return 0
    if args.case == "sec4":
        print(json.dumps({"case": "sec4", **sec4_case()}), flush=True)
        return 0
    if args.case == "series-profile":
        return series_case()
    if args.case == "geometry":
        print(json.dumps({"case": "geometry", **geometry_case()}), flush=True)
        return 0
    if args.case == "offdiag":
        print(json.dumps({"case": "offdiag", **offdiag_case()}), flush=True)
        return 0
    if args.case == "spectrum-dns":
        print(json.dumps({"case": "spectrum-dns", **spectrum_dns_case()}), flush=True)
        return 0

    import torch
    import torch.distributed as dist
    import paper_1510_00451_gb300 as mlsd

    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    torch.cuda.set_device(_local_rank())
    dev = torch.device("cuda", _local_rank())
    if world > 1:
        dist.init_process_group("nccl", device_id=dev)

    def barrier():
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize()

    cfg = _workload()
    N, L = cfg["n_macro"], len(cfg["patch_n"])
    stream = torch.cuda.current_stream()
    lv = mlsd.Levels(cfg["spectrum"], cfg["kappa"], N, cfg["edges"], cfg["patch_n"],
                     cfl=cfg["cfl"], t_burn_tau=8.0, t_avg_tau=4.0, precision=cfg["precision"])
    K = torch.zeros(N * N, 3, dtype=torch.float64, device=dev)
    U0 = torch.tensor(__import__("inputs").gaussian_u0(N, cfg["sigma"]), dtype=torch.float32,
                      device=dev)
    U = torch.empty_like(U0)
    flush = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)  # > L2 (129 MB)

    def step():
        lv.effective_diffusivity(K)
        dt = mlsd.macro_dt(K, N, cfg["cfl"])
        ns = max(1, math.ceil(cfg["T"] / dt))
        U.copy_(U0)
        mlsd.macro_step(U, K, cfg["T"] / ns, ns, want_mass=False)

    for _ in range(args.warmup):
        step()
    assert lv.status() == 0
    work = [lv.level_work(l + 1) for l in range(L)]
    cell_updates = sum(w[0] for w in work)
    window_updates = sum(w[2] for w in work)

    # ---- timed region: K steps, device time per step (L2 flushed between steps)
    clk_path = tempfile.mktemp(prefix="mlsd_clocks_", suffix=".csv")
    sampler = _clock_sampler(clk_path)
    for l in range(L):
        lv.profile_collect(l + 1)          # drop warm-up events
    lv.profile(True)
    launches0 = mlsd.launch_count()
    evs = []
    barrier()
    t_wall = time.perf_counter()
    for _ in range(args.steps):
        flush.zero_()
        e0 = torch.cuda.Event(enable_timing=True); e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        step()
        e1.record(stream)
        evs.append((e0, e1))
    barrier()
    t_wall = time.perf_counter() - t_wall
    launches = mlsd.launch_count() - launches0
    lv.profile(False)
    if sampler:
        sampler.terminate(); sampler.wait()
    clocks = _clock_summary(clk_path)
    ms_step = sum(a.elapsed_time(b) for a, b in evs) / args.steps
    kern_ms, kern_n = 0.0, 0
    per_level = []
    for l in range(L):
        ms, n = lv.profile_collect(l + 1)
        kern_ms += ms; kern_n += n
        cu_l = work[l][0]
        per_level.append({"level": l + 1, "kernel_ms_per_step": ms / args.steps,
                          "cell_updates": cu_l, "max_steps_per_patch": work[l][1],
                          "cell_updates_per_s": cu_l / (ms / args.steps * 1e-3) if ms > 0 else None,
                          "k_eff_tensors_per_s": N * N / (ms / args.steps * 1e-3) if ms > 0 else None})
    kern_ops = args.steps * (cell_updates * OPS_PER_CELL_UPDATE
                             + window_updates * OPS_PER_WINDOW_UPDATE)
    kern_flop = args.steps * (cell_updates * FLOP_PER_CELL_UPDATE
                              + window_updates * FLOP_PER_WINDOW_UPDATE)
    assert lv.status() == 0
    ms_step = ranks_max(ms_step, world, dev)
    value = job_rate(cell_updates, ms_step, world)
    tensors = job_rate(N * N, ms_step, world)

    # ---- end to end through the C ABI with host buffers (pinned)
    e2e = None
    if not args.no_e2e:
        U0_h = U0.cpu().pin_memory()
        K_h = torch.empty(N * N, 3, dtype=torch.float64).pin_memory()
        U_h = torch.empty(N, N, dtype=torch.float32).pin_memory()
        Ud = torch.empty_like(U0)
        barrier()
        e0 = torch.cuda.Event(enable_timing=True); e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(args.steps):
            Ud.copy_(U0_h, non_blocking=True)
            lv.effective_diffusivity(K)
            dt = mlsd.macro_dt(K, N, cfg["cfl"])
            ns = max(1, math.ceil(cfg["T"] / dt))
            mlsd.macro_step(Ud, K, cfg["T"] / ns, ns, want_mass=False)
            K_h.copy_(K, non_blocking=True)
            U_h.copy_(Ud, non_blocking=True)
        e1.record(stream)
        barrier()
        ms_e2e = ranks_max(e0.elapsed_time(e1) / args.steps, world, dev)
        e2e = {"value": job_rate(cell_updates, ms_e2e, world), "unit": UNIT,
               "h2d_bytes_per_step": U0_h.numel() * 4,
               "d2h_bytes_per_step": K_h.numel() * 8 + U_h.numel() * 4}

    dns = None
    if not args.no_dns:
        d = dns_case(8192, 1000)
        gbs = DNS_BYTES_PER_CELL_STEP * d["cell_steps_per_s"] / 1e9
        hbm, hbm_src = _peak("hbm_gbs")
        dns = {"workload": "continuous_spectrum_dns (8192^2 FP32, |k|<=256, kappa=1e-3, 1000 steps)",
               "value": d["cell_steps_per_s"] * world, "unit": "cell-steps/s", "ms": d["ms"],
               "roofline": {"bound": "hbm", "achieved": gbs, "peak": hbm, "peak_source": hbm_src,
                            "unit": "GB/s",
                            "frac": gbs / hbm, "traffic": DNS_DRAM_BYTES_PER_LAUNCH.get(d["kernel"]),
                            "traffic_unit": "DRAM bytes per launch (ncu, 8192^2)",
                            "kernel": d["kernel"],
                            "algorithmic_bytes_per_cell_step": DNS_BYTES_PER_CELL_STEP},
               "mass_rel_drift": d["mass_rel_drift"], "finite": d["finite"]}

    sur = None
    if not args.no_surrogate:
        sur = surrogate_case()
    unev = None
    if not args.no_uneven:
        unev = uneven_case()
    experiments = None
    if not args.no_experiments and rank == 0:
        experiments = {}
        for name, fn in (("sec4_setup", sec4_case), ("offdiag_stress", offdiag_case),
                         ("patch_geometry", geometry_case)):
            try:
                experiments[name] = fn()
            except Exception as exc:           # reported in the line, not fatal to it
                experiments[name] = {"error": repr(exc)}

    if rank != 0:
        if world > 1:
            dist.destroy_process_group()
        return 0

    line_extra = {}
    peaks = _peaks()
    sm_count = torch.cuda.get_device_properties(dev).multi_processor_count
    sm_max = peaks.get("sm_max_mhz", 2070.0)
    issue_peak = sm_count * 128 * sm_max * 1e6 / 1e12             # T FP32 instructions/s
    flop_peak = 2 * issue_peak                                     # TFLOP/s, all FFMA
    achieved = kern_ops / (kern_ms * 1e-3) / 1e12 if kern_ms > 0 else None
    achieved_flop = kern_flop / (kern_ms * 1e-3) / 1e12 if kern_ms > 0 else None
    cpu = None
    if not args.no_cpu_baseline and world == 1:
        import oracle
        cores = oracle.num_threads()
        v, secs, sample, nodes, Kor = _oracle_sample(cores)
        cpu = {"value": v, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": sample,
               "seconds": secs}
        Kg = K.cpu().numpy()
        errs = [float(np.linalg.norm(Kg[j * N + i] - Kor[t]) / np.linalg.norm(Kor[t]))
                for t, (i, j) in enumerate(nodes)]
        line_extra["k_eff_rel_err_vs_oracle"] = {"max": max(errs), "nodes": len(nodes)}
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": _config(world),
        "k_eff_tensors_per_s": tensors,
        "cell_updates_per_step": cell_updates * world,
        "per_level": per_level,
        "roofline": {"bound": "alu", "achieved": achieved, "peak": issue_peak,
                     "unit": "T FP32-pipe instructions/s",
                     "frac": (achieved / issue_peak) if achieved else None,
                     "traffic": PATCH_DRAM_BYTES_PER_LAUNCH,
                     "traffic_unit": "DRAM bytes per launch (ncu), against 0 algorithmic",
                     "kernel": "k_patch_solve", "launches": kern_n,
                     "kernel_ms_per_step": kern_ms / args.steps,
                     "algorithmic": f"{OPS_PER_CELL_UPDATE} FP32 FADD/FMUL/FFMA per cell-update "
                                    f"+ {OPS_PER_WINDOW_UPDATE} per averaging-window cell-update",
                     "window_fraction": window_updates / cell_updates,
                     "peak_basis": f"{sm_count} SMs x 128 FP32 lanes x {sm_max:.0f} MHz, one "
                                   "FADD/FMUL/FFMA per lane per clock",
                     "flop": {"achieved": achieved_flop, "peak": flop_peak, "unit": "TFLOP/s",
                              "frac": (achieved_flop / flop_peak) if achieved_flop else None,
                              "per_cell_update": f"{FLOP_PER_CELL_UPDATE} + {FLOP_PER_WINDOW_UPDATE}"
                                                 " in the window"}},
        "cpu_baseline": cpu,
        "e2e": e2e,
        "clocks": clocks,
        "gpu_launches": launches,
        "wall_s_timed": t_wall,
        "dns": dns,
        "surrogate": sur,
        "uneven_sizes": unev,
        "experiments": experiments,
    }
    line.update(line_extra)
    print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
