"""FP64 CPU oracle of the multiscale effective-diffusivity method.

TEST INFRASTRUCTURE ONLY: imported by tests/, by the smoke check and by the
CPU-baseline leg of the benchmark, never by the library.  Every function is a
thin ctypes wrapper over oracle/mlsd_oracle.c; the arithmetic lives there and
each C routine cites the section or algorithm of the paper it follows.

Pins: the closed forms and invariants that fix each routine are exercised by
tests/test_oracle_*.py (shear closed form, transient closed form, direct
steady solve, Proposition 1, Algorithm 1 on shears, Fourier amplification of
the macro scheme, conservation, symmetry, kappa-only limit).
"""
import ctypes
import math
import os

import numpy as np

from . import build as _build

_lib = None


def lib():
    global _lib
    if _lib is None:
        _build.build()
        _lib = ctypes.CDLL(_build.LIB)
        _declare(_lib)
    return _lib


_i = ctypes.c_int
_l = ctypes.c_long
_d = ctypes.c_double
_p = ctypes.c_void_p


def _declare(L):
    L.orc_band_of.argtypes = [_i, _p, _p, _i, _p, _p, _p]
    L.orc_patch_origin.argtypes = [_i, _i, _l, _i]
    L.orc_patch_origin.restype = _l
    L.orc_patch_psi.argtypes = [_i, _p, _p, _p, _p, _p, _l, _l, _l, _i, _p]
    L.orc_velocity.argtypes = [_i, _d, _p, _p, _p]
    L.orc_lambda_min.argtypes = [_p]
    L.orc_lambda_min.restype = _d
    L.orc_micro_dt.argtypes = [_d, _d, _p, _d]
    L.orc_micro_dt.restype = _d
    L.orc_micro_steps.argtypes = [_d, _p, _d, _d, _d, _p, _p]
    L.orc_corrector_rhs.argtypes = [_i, _d, _p, _p, _i, _p, _p]
    L.orc_patch_k.argtypes = [_i, _d, _p, _p, _d, _l, _l, _p, _p, _p]
    L.orc_corrector_energy.argtypes = [_i, _d, _p, _p, _p, _p]
    L.orc_offdiag_q.argtypes = [_i, _p, _p, _p, _p, _p, _p, _l, _l, _l, _i, _d, _p, _p]
    L.orc_offdiag_apply.argtypes = [_i, _p, _p, _p, _p]
    L.orc_chain.argtypes = [_i, _p, _p, _p, _p, _i, _p, _p, _p, _i, _d, _d, _d, _d, _l, _l,
                            _i, _p, _p, _p, _p, _p, _i]
    L.orc_patch_n_rule.argtypes = [_i, _p, _p, _p, _p, _p, _l, _i, _i, _i, _d, _i, _i, _i, _p]
    L.orc_patch_n_rule.restype = _i
    L.orc_macro_dt.argtypes = [_i, _p, _d]
    L.orc_macro_dt.restype = _d
    L.orc_macro_run.argtypes = [_i, _p, _p, _d, _l, _p]
    L.orc_dns_run.argtypes = [_i, _p, _d, _d, _l, _p]
    L.orc_macro_run_dirichlet.argtypes = [_i, _p, _p, _d, _l, _d, _d]
    L.orc_dns_run_dirichlet.argtypes = [_i, _p, _d, _d, _l, _d, _d, _p]
    L.orc_grid_psi.argtypes = [_i, _p, _p, _p, _p, _i, _p]
    L.orc_coarse_grain.argtypes = [_i, _p, _i, _p, _p]
    L.orc_num_threads.restype = _i
    L.orc_features.argtypes = [_i, _p, _p, _d, _p]
    L.orc_series.argtypes = [_i, _d, _p, _p, _i, _p]
    L.orc_series_estimate.argtypes = [_p, _p, _p, _p, _p]
    L.orc_wynn.argtypes = [_p, _i, _i]
    L.orc_wynn.restype = _d
    L.orc_periodic_smooth.argtypes = [_i, _p, _p]
    L.orc_mlp.argtypes = [_i, _i, _i, _p, _p, _i, _p, _p, _p]
    L.orc_mlp.restype = _d


def _ptr(a):
    return None if a is None else a.ctypes.data


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def _i32(a):
    return np.ascontiguousarray(a, dtype=np.int32)


def num_threads():
    return lib().orc_num_threads()


def _modes(spec):
    return (_i32(spec.k1), _i32(spec.k2), _f64(spec.re), _f64(spec.im))


def band_of(spec, edges):
    """Per mode: (level 1..L or -1, kind 0 diag / 1 psi_12 / 2 psi_21 / -1)."""
    k1, k2, re, im = _modes(spec)
    e = _f64(edges)
    lev = np.zeros(len(k1), np.int32)
    kind = np.zeros(len(k1), np.int32)
    lib().orc_band_of(len(k1), _ptr(k1), _ptr(k2), len(e) - 1, _ptr(e), _ptr(lev), _ptr(kind))
    return lev, kind


def patch_origin(i, n_macro, Nl, n):
    return lib().orc_patch_origin(int(i), int(n_macro), int(Nl), int(n))


def patch_psi(spec, Nl, ox, oy, n, use=None):
    k1, k2, re, im = _modes(spec)
    u = None if use is None else np.ascontiguousarray(use, dtype=np.uint8)
    psi = np.zeros((n, n))
    lib().orc_patch_psi(len(k1), _ptr(k1), _ptr(k2), _ptr(re), _ptr(im), _ptr(u),
                        int(Nl), int(ox), int(oy), int(n), _ptr(psi))
    return psi


def velocity(psi, h):
    psi = _f64(psi)
    n = psi.shape[0]
    v1 = np.zeros((n, n)); v2 = np.zeros((n, n))
    lib().orc_velocity(n, float(h), _ptr(psi), _ptr(v1), _ptr(v2))
    return v1, v2


def lambda_min(B):
    B = _f64(B)
    return lib().orc_lambda_min(_ptr(B))


def micro_dt(h, vmax, B, cfl):
    B = _f64(B)
    return lib().orc_micro_dt(float(h), float(vmax), _ptr(B), float(cfl))


def micro_steps(L, B, dt, t_burn=8.0, t_avg=4.0):
    nb = ctypes.c_long(); na = ctypes.c_long()
    B = _f64(B)
    lib().orc_micro_steps(float(L), _ptr(B), float(dt), float(t_burn), float(t_avg),
                          ctypes.byref(nb), ctypes.byref(na))
    return nb.value, na.value


def corrector_rhs(psi, h, B, j, w):
    psi = _f64(psi); w = _f64(w); B = _f64(B)
    f = np.zeros_like(w)
    lib().orc_corrector_rhs(psi.shape[0], float(h), _ptr(psi), _ptr(B), int(j), _ptr(w), _ptr(f))
    return f


def patch_k(psi, h, B, dt, n_burn, n_avg, want_w=False, want_S=False):
    """K[psi, B; D] of one patch: returns K (3,), and optionally w (2, n, n), S (4,)."""
    psi = _f64(psi); B = _f64(B)
    n = psi.shape[0]
    K = np.zeros(3)
    w = np.zeros((2, n, n)) if want_w else None
    S = np.zeros(4) if want_S else None
    lib().orc_patch_k(n, float(h), _ptr(psi), _ptr(B), float(dt), int(n_burn), int(n_avg),
                      _ptr(K), _ptr(w), _ptr(S))
    out = [K]
    if want_w:
        out.append(w)
    if want_S:
        out.append(S)
    return out[0] if len(out) == 1 else tuple(out)


def corrector_energy(w, h, B):
    """Energy form E (E11, E12, E22) and the means of the corrector pair w[2][n][n]."""
    w = _f64(w); B = _f64(B)
    E = np.zeros(3); m = np.zeros(2)
    lib().orc_corrector_energy(w.shape[1], float(h), _ptr(w), _ptr(B), _ptr(E), _ptr(m))
    return E, m


def offdiag_q(spec, use12, use21, Nl, ox, oy, n, L):
    k1, k2, re, im = _modes(spec)
    q12 = np.zeros(n); q21 = np.zeros(n)
    u12 = np.ascontiguousarray(use12, np.uint8)
    u21 = np.ascontiguousarray(use21, np.uint8)
    lib().orc_offdiag_q(len(k1), _ptr(k1), _ptr(k2), _ptr(re), _ptr(im), _ptr(u12), _ptr(u21),
                        int(Nl), int(ox), int(oy), int(n), float(L), _ptr(q12), _ptr(q21))
    return q12, q21


def offdiag_apply(q12, q21, B):
    """Algorithms 1-2 from line variances; pass None for a part the level lacks."""
    q12 = None if q12 is None else _f64(q12)
    q21 = None if q21 is None else _f64(q21)
    B = _f64(B)
    n = len(q12) if q12 is not None else (len(q21) if q21 is not None else 1)
    out = np.zeros(3)
    lib().orc_offdiag_apply(n, _ptr(q12), _ptr(q21), _ptr(B), _ptr(out))
    return out


def level_lattice(edges, patch_n, patch_div=None):
    """Lattice size Nl = n * m_l per level; L_l = 2 pi / m_l with m_l = e_{l-1}
    by default (one period of the level's lowest wavenumber)."""
    Lc = len(edges) - 1
    m = level_div(edges, patch_div)
    return [int(patch_n[l]) * m[l] for l in range(Lc)]


def level_div(edges, patch_div=None):
    Lc = len(edges) - 1
    if patch_div is None:
        return [int(round(edges[l])) for l in range(Lc)]
    return [int(x) for x in patch_div]


def patch_n_rule(spec, edges, level, node, n_macro, kappa, n_min=32, n_max=256, nref=32,
                 patch_div=None):
    """Patch resolution of one node at one level (uneven patch sizes)."""
    k1, k2, re, im = _modes(spec)
    lev, kind = band_of(spec, edges)
    use = np.ascontiguousarray((lev == level) & (kind == 0), dtype=np.uint8)
    m = level_div(edges, patch_div)[level - 1]
    vm = ctypes.c_double()
    n = lib().orc_patch_n_rule(len(k1), _ptr(k1), _ptr(k2), _ptr(re), _ptr(im), _ptr(use), int(m),
                               int(node[0]), int(node[1]), int(n_macro), float(kappa), int(nref),
                               int(n_min), int(n_max), ctypes.byref(vm))
    return n, vm.value


def chain(spec, edges, patch_n, n_macro, kappa, nodes, cfl=0.2, t_burn=8.0, t_avg=4.0,
          n_burn_fixed=-1, n_avg_fixed=0, patch_div=None, want_levels=False, want_steps=False,
          node_n=None, periodize=False):
    """Algorithm 3 down the whole level hierarchy for the macro nodes (i, j) given.

    patch_n gives n per level; node_n (optional, [nodes][L]) overrides it per node.
    Returns K [nodes][3]; with want_levels also K*_l [nodes][L][3]; with want_steps
    also the step counts n_burn + n_avg [nodes][L] of every patch solve."""
    k1, k2, re, im = _modes(spec)
    e = _f64(edges)
    Lc = len(e) - 1
    nodes = np.asarray(nodes, dtype=np.int32).reshape(-1, 2)
    ni = _i32(nodes[:, 0]); nj = _i32(nodes[:, 1])
    if node_n is None:
        node_n = np.tile(np.asarray(patch_n, dtype=np.int32), (len(ni), 1))
    nn = np.ascontiguousarray(node_n, dtype=np.int32).reshape(len(ni), Lc)
    md = np.ascontiguousarray(level_div(edges, patch_div), dtype=np.int64)
    K = np.zeros((len(ni), 3))
    Kl = np.zeros((len(ni), Lc, 3)) if want_levels else None
    st = np.zeros((len(ni), Lc), dtype=np.int64) if want_steps else None
    lib().orc_chain(len(k1), _ptr(k1), _ptr(k2), _ptr(re), _ptr(im), Lc, _ptr(e), _ptr(nn),
                    _ptr(md), int(n_macro), float(kappa), float(cfl), float(t_burn), float(t_avg),
                    int(n_burn_fixed), int(n_avg_fixed), len(ni), _ptr(ni), _ptr(nj),
                    _ptr(K), _ptr(Kl), _ptr(st), 1 if periodize else 0)
    out = [K]
    if want_levels:
        out.append(Kl)
    if want_steps:
        out.append(st)
    return out[0] if len(out) == 1 else tuple(out)


def macro_dt(K, n_macro, cfl):
    K = _f64(K)
    return lib().orc_macro_dt(int(n_macro), _ptr(K), float(cfl))


def macro_run(U, K, dt, nsteps, want_mass=True):
    U = _f64(U).copy(); K = _f64(K)
    N = U.shape[0]
    mass = np.zeros(nsteps + 1) if want_mass else None
    lib().orc_macro_run(N, _ptr(U), _ptr(K), float(dt), int(nsteps), _ptr(mass))
    return (U, mass) if want_mass else U


def grid_psi(spec, Nf):
    k1, k2, re, im = _modes(spec)
    psi = np.zeros((Nf, Nf))
    lib().orc_grid_psi(len(k1), _ptr(k1), _ptr(k2), _ptr(re), _ptr(im), int(Nf), _ptr(psi))
    return psi


def dns_run(psi, kappa, dt, nsteps, u0):
    psi = _f64(psi); u = _f64(u0).copy()
    lib().orc_dns_run(psi.shape[0], _ptr(psi), float(kappa), float(dt), int(nsteps), _ptr(u))
    return u


def macro_run_dirichlet(U, K, dt, nsteps, u_left=1.0, u_right=0.0):
    """Macro steps with the Sec. 4 boundaries: Dirichlet in x1 (column 0 held at
    u_left, the virtual column N at u_right), periodic in x2.  Returns U."""
    U = _f64(U).copy(); K = _f64(K)
    N = U.shape[0]
    lib().orc_macro_run_dirichlet(N, _ptr(U), _ptr(K), float(dt), int(nsteps), float(u_left),
                                  float(u_right))
    return U


def dns_run_dirichlet(psi, kappa, dt, nsteps, u0, u_left=1.0, u_right=0.0):
    """Direct simulation with the Sec. 4 boundaries (as macro_run_dirichlet)."""
    psi = _f64(psi); u = _f64(u0).copy()
    lib().orc_dns_run_dirichlet(psi.shape[0], _ptr(psi), float(kappa), float(dt), int(nsteps),
                                float(u_left), float(u_right), _ptr(u))
    return u


def coarse_grain(u, N):
    u = _f64(u)
    U = np.zeros((N, N)); m = ctypes.c_double()
    lib().orc_coarse_grain(u.shape[0], _ptr(u), int(N), _ptr(U), ctypes.byref(m))
    return U, m.value


N_FEATURES = 606
SERIES_M = 19
PSI_SCALE, T_SCALE, Y_SCALE = 32.0, 10.0, 300.0


def features(psi, B, kappa):
    """606 surrogate inputs of one patch (psi with its patch mean removed); a patch
    above 64 x 64 is described by its samples on the 64 x 64 sub-lattice."""
    psi = _f64(psi); B = _f64(B)
    f = np.zeros(N_FEATURES)
    lib().orc_features(psi.shape[0], _ptr(psi), _ptr(B), float(kappa), _ptr(f))
    return f


def periodic_smooth(u):
    """Periodic component p of an n x n patch field (u = p + s, Moisan 2011)."""
    u = _f64(u)
    p = np.zeros_like(u)
    lib().orc_periodic_smooth(u.shape[0], _ptr(u), _ptr(p))
    return p


def series(psi, B, M=SERIES_M, h=None):
    """Perturbation moments T_2..T_M of the steady corrector equation: [M-1][3]
    (components 11, 12, 22); sum_m T_m = K - B where the series converges."""
    psi = _f64(psi); B = _f64(B)
    n = psi.shape[0]
    T = np.zeros((M - 1, 3))
    lib().orc_series(n, float(2 * np.pi / n if h is None else h), _ptr(psi), _ptr(B), int(M),
                     _ptr(T))
    return T


def wynn(T, comp, K):
    """[K/K] Pade value at 1 of the series in x^2 with terms T_(2k+2) + T_(2k+3)
    (Wynn's epsilon on its partial sums)."""
    T = _f64(T)
    return lib().orc_wynn(_ptr(T), int(comp), int(K))


def series_estimate(T):
    """(P2, P3, E, gap): the [2/2], [3/3], [4/4] approximants of K - B from
    T_2..T_19 and the gap max_c |E_c - P3_c|."""
    T = _f64(T)
    P2 = np.zeros(3); P3 = np.zeros(3); E = np.zeros(3); gap = ctypes.c_double()
    lib().orc_series_estimate(_ptr(T), _ptr(P2), _ptr(P3), _ptr(E), ctypes.byref(gap))
    return P2, P3, E, gap.value


def surrogate_target(K, B, E):
    """Training target of one patch: asinh((K - B - E) Y_SCALE / tr B)."""
    return np.arcsinh((np.asarray(K) - np.asarray(B) - np.asarray(E)) * Y_SCALE / (B[0] + B[2]))


def surrogate_K(out, E, B):
    """K of one patch from a network output and the series estimate E."""
    return np.asarray(B) + np.asarray(E) + (B[0] + B[2]) * np.sinh(np.asarray(out)) / Y_SCALE


def mlp_param_count(d0, h):
    return h * d0 + h + 2 * (h * h + h) + 3 * h + 3


def mlp(X, params, h, bf16=True, Y=None, want_grad=False):
    """FP64 forward (and loss / gradient) of one surrogate member."""
    X = _f64(X); params = _f64(params)
    M, d0 = X.shape
    assert params.size == mlp_param_count(d0, h)
    out = np.zeros((M, 3))
    Yc = None if Y is None else _f64(Y)
    g = np.zeros_like(params) if want_grad else None
    loss = lib().orc_mlp(M, d0, h, _ptr(X), _ptr(params), 1 if bf16 else 0, _ptr(Yc), _ptr(out), _ptr(g))
    if Y is None:
        return out
    return (out, loss, g) if want_grad else (out, loss)
