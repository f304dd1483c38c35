"""Helpers shared by the GPU parity tests: oracle values for selected patches.

Only the oracle computes expected values; the CUDA path is never an input.
"""
import math
from concurrent.futures import ThreadPoolExecutor

import numpy as np

import oracle


def rel_l2(a, b):
    a = np.asarray(a, dtype=np.float64); b = np.asarray(b, dtype=np.float64)
    den = np.linalg.norm(b)
    return np.linalg.norm(a - b) / (den if den > 0 else 1.0)


def level_geometry(edges, patch_n, level, patch_div=None):
    Nl = oracle.level_lattice(edges, patch_n, patch_div)[level - 1]
    n = patch_n[level - 1]
    h = 2 * math.pi / Nl
    return n, Nl, h, n * h


def oracle_level(spec, edges, patch_n, level, n_macro, B, patches, cfl=0.2, t_burn=8.0,
                 t_avg=4.0, n_burn_fixed=-1, n_avg_fixed=0, want_w=False, workers=8):
    """Oracle K (and optionally w) of the given patches of one level with base B[p]."""
    lev, kind = oracle.band_of(spec, edges)
    use = (lev == level) & (kind == 0)
    n, Nl, h, L = level_geometry(edges, patch_n, level)

    def one(p):
        i, j = p % n_macro, p // n_macro
        ox = oracle.patch_origin(i, n_macro, Nl, n)
        oy = oracle.patch_origin(j, n_macro, Nl, n)
        psi = oracle.patch_psi(spec, Nl, ox, oy, n, use=use)
        v1, v2 = oracle.velocity(psi, h)
        vmax = float(np.max(np.abs(v1) + np.abs(v2)))
        Bp = np.asarray(B[p], dtype=np.float64)
        dt = oracle.micro_dt(h, vmax, Bp, cfl)
        if n_avg_fixed > 0:
            nb, na = n_burn_fixed, n_avg_fixed
        else:
            nb, na = oracle.micro_steps(L, Bp, dt, t_burn, t_avg)
        return oracle.patch_k(psi, h, Bp, dt, nb, na, want_w=want_w)

    with ThreadPoolExecutor(workers) as ex:
        return list(ex.map(one, patches))


def random_spd(P, rng, lo=0.02, hi=0.08):
    a = rng.uniform(lo, hi, (P, 2))
    c = rng.uniform(-0.4, 0.4, P) * np.sqrt(a[:, 0] * a[:, 1])
    return np.stack([a[:, 0], c, a[:, 1]], 1)


def square_symmetry_psi(psi, g):
    """Patch samples psi[b][a] (b along x2, a along x1) under element g of the
    square's symmetry group: bit 0 reflects x1 (a -> -a mod n), bit 1 reflects
    x2, bit 2 then swaps x1 and x2.  Each reflection or swap negates psi, as a
    stream function is a pseudo-scalar, so that v maps as a vector."""
    out = np.asarray(psi, dtype=np.float64)
    if g & 1:
        out = -np.roll(out[:, ::-1], 1, axis=1)
    if g & 2:
        out = -np.roll(out[::-1, :], 1, axis=0)
    if g & 4:
        out = -out.T
    return np.ascontiguousarray(out)


def square_symmetry_tensor(T, g):
    """Symmetric tensor (T11, T12, T22) under the same element: R T R^T with R
    the product of the element's reflections and swap."""
    R = np.eye(2)
    if g & 1:
        R = np.diag([-1.0, 1.0]) @ R
    if g & 2:
        R = np.diag([1.0, -1.0]) @ R
    if g & 4:
        R = np.array([[0.0, 1.0], [1.0, 0.0]]) @ R
    M = R @ np.array([[T[0], T[1]], [T[1], T[2]]], dtype=np.float64) @ R.T
    return np.array([M[0, 0], M[0, 1], M[1, 1]])
