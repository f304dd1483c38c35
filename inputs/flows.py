"""Seeded synthetic stream functions and initial conditions.

A stream function is given by a Hermitian-complete list of Fourier modes
(k1, k2, re, im) on the periodic domain [0, 2*pi)^2:

    psi(x) = sum_modes Re[(re + i*im) * exp(i*(k1*x1 + k2*x2))]

so that the list for a real field holds every mode together with its mirror
-k carrying the complex-conjugate coefficient.  The flows below follow the
shapes of the paper's examples (Sec. 4.2 cellular modes, Sec. 4.4 continuous
spectrum) at the sizes of the workloads this library is measured on.
"""
from dataclasses import dataclass, field
import math

import numpy as np


@dataclass
class Spectrum:
    k1: np.ndarray
    k2: np.ndarray
    re: np.ndarray
    im: np.ndarray
    meta: dict = field(default_factory=dict)

    @property
    def n_modes(self):
        return int(self.k1.shape[0])

    def as_arrays(self):
        return (np.ascontiguousarray(self.k1, dtype=np.int32),
                np.ascontiguousarray(self.k2, dtype=np.int32),
                np.ascontiguousarray(self.re, dtype=np.float64),
                np.ascontiguousarray(self.im, dtype=np.float64))


def _from_dict(d, meta=None):
    keys = sorted(d)
    k1 = np.array([k[0] for k in keys], dtype=np.int32)
    k2 = np.array([k[1] for k in keys], dtype=np.int32)
    re = np.array([d[k].real for k in keys], dtype=np.float64)
    im = np.array([d[k].imag for k in keys], dtype=np.float64)
    return Spectrum(k1, k2, re, im, meta or {})


def _add(d, k, c):
    d[k] = d.get(k, 0.0) + c


def _add_sinsin(d, a, m1, m2):
    """a * sin(m1 x1) sin(m2 x2) as Hermitian mode pairs.

    sin(p)sin(q) = [cos(p - q) - cos(p + q)] / 2 and cos(t) = (e^{it} + e^{-it}) / 2.
    """
    _add(d, (m1, -m2), a / 4)
    _add(d, (-m1, m2), a / 4)
    _add(d, (m1, m2), -a / 4)
    _add(d, (-m1, -m2), -a / 4)


def cellular_two_scale(a0=1.0, a1=1.0, m=8):
    """psi = a0 sin x sin y + a1 sin(m x) sin(m y): two-scale cellular flow."""
    d = {}
    _add_sinsin(d, a0, 1, 1)
    _add_sinsin(d, a1, m, m)
    return _from_dict(d, {"kind": "cellular_two_scale", "m": m})


def cellular(terms):
    """psi = sum over (a, m1, m2) of a sin(m1 x1) sin(m2 x2) (the paper's phi_c
    cellular modes, Sec. 4.2 / 4.3, on [0, 2 pi)^2)."""
    d = {}
    for a, m1, m2 in terms:
        _add_sinsin(d, a, m1, m2)
    return _from_dict(d, {"kind": "cellular", "terms": list(terms)})


def cellular_hierarchy(levels=3, alpha=4):
    """psi = sum_j alpha^-j sin(alpha^j x) sin(alpha^j y), j = 0..levels-1."""
    d = {}
    for j in range(levels):
        _add_sinsin(d, float(alpha) ** (-j), alpha ** j, alpha ** j)
    return _from_dict(d, {"kind": "cellular_hierarchy", "alpha": alpha})


def shear_x1(amp, m, phase=0.0):
    """psi = amp * sin(m x1 + phase): a shear flow v = (0, v2(x1))."""
    # sin(t) = (e^{it} - e^{-it}) / (2i): coefficient of e^{i m x1} is -i e^{i phase} / 2
    c = -0.5j * complex(math.cos(phase), math.sin(phase)) * amp
    d = {(m, 0): c, (-m, 0): c.conjugate()}
    return _from_dict(d, {"kind": "shear_x1"})


def shear_x2(amp, m, phase=0.0):
    """psi = amp * sin(m x2 + phase): a shear flow v = (v1(x2), 0)."""
    c = -0.5j * complex(math.cos(phase), math.sin(phase)) * amp
    d = {(0, m): c, (0, -m): c.conjugate()}
    return _from_dict(d, {"kind": "shear_x2"})


def shear_diag(amp, m):
    """psi = amp * sin(m (x1 + x2)): a shear along the diagonal."""
    c = -0.5j * amp
    d = {(m, m): c, (-m, -m): c.conjugate()}
    return _from_dict(d, {"kind": "shear_diag"})


def combine(*spectra):
    d = {}
    for s in spectra:
        for a, b, r, i in zip(s.k1, s.k2, s.re, s.im):
            _add(d, (int(a), int(b)), complex(r, i))
    return _from_dict(d, {"kind": "combined"})


_MASK64 = (1 << 64) - 1


def splitmix64(seed, count):
    """SplitMix64 stream (Steele, Lea & Flood 2014), `count` uint64 outputs."""
    out = np.empty(count, dtype=np.uint64)
    x = seed & _MASK64
    for t in range(count):
        x = (x + 0x9E3779B97F4A7C15) & _MASK64
        z = x
        z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & _MASK64
        z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & _MASK64
        out[t] = z ^ (z >> 31)
    return out


def continuous_spectrum(kmax=256, seed=1510004510, slope=-7.0 / 3.0, vrms=1.0):
    """Random-phase stream function with every integer mode 1 <= |k| <= kmax.

    |psi_hat(k)| ~ |k|^slope; slope = -7/3 gives a shell energy spectrum
    E(k) ~ k * k^2 |psi_hat|^2 ~ k^(-5/3).  Phases are uniform on [0, 2 pi)
    from SplitMix64(seed), drawn once per mode of the upper half plane
    (k2 > 0, or k2 == 0 and k1 > 0) in order of increasing k2 then k1; the
    mirror mode gets the conjugate.  The field is scaled so that the rms
    speed sum_k |k|^2 |psi_hat(k)|^2 equals vrms^2.
    """
    half = []
    for k2 in range(0, kmax + 1):
        for k1 in range(-kmax, kmax + 1):
            if k2 == 0 and k1 <= 0:
                continue
            r2 = k1 * k1 + k2 * k2
            if 1 <= r2 <= kmax * kmax:
                half.append((k1, k2))
    u = splitmix64(seed, len(half))
    phase = (u >> np.uint64(11)).astype(np.float64) * (2.0 ** -53) * 2.0 * math.pi
    kk = np.array(half, dtype=np.int64)
    kabs = np.sqrt((kk ** 2).sum(1).astype(np.float64))
    amp = kabs ** slope
    # rms speed^2 = sum over the full Hermitian set of |k|^2 |c|^2 = 2 * half-plane sum
    e = 2.0 * np.sum(kabs ** 2 * amp ** 2)
    amp = amp * (vrms / math.sqrt(e))
    re = amp * np.cos(phase)
    im = amp * np.sin(phase)
    k1 = np.concatenate([kk[:, 0], -kk[:, 0]]).astype(np.int32)
    k2 = np.concatenate([kk[:, 1], -kk[:, 1]]).astype(np.int32)
    return Spectrum(k1, k2, np.concatenate([re, re]), np.concatenate([im, -im]),
                    {"kind": "continuous_spectrum", "kmax": kmax, "seed": seed})


def gaussian_u0(n, sigma=0.5, center=(math.pi, math.pi), dtype=np.float64):
    """U0 = exp(-|x - c|^2 / (2 sigma^2)) on the n x n node grid of [0, 2pi)^2,
    with the minimum-image distance; array layout [j][i] (x2 slow, x1 fast)."""
    x = 2.0 * math.pi * np.arange(n) / n
    def dist(a, c):
        d = np.abs(a - c)
        return np.minimum(d, 2.0 * math.pi - d)
    dx = dist(x, center[0])[None, :]
    dy = dist(x, center[1])[:, None]
    return np.exp(-(dx ** 2 + dy ** 2) / (2.0 * sigma ** 2)).astype(dtype)


def step_u0(n, u_left=1.0, u_right=0.0, dtype=np.float64):
    """The step initial condition of the Sec. 4 set-up on [0, 2 pi] x [0, 2 pi):
    u0 = u_left for x1 <= pi, u_right for x1 > pi, on the n x n node grid
    x1 = 2 pi i / n (column 0 is the boundary x1 = 0); layout [j][i]."""
    x = 2.0 * math.pi * np.arange(n) / n
    row = np.where(x <= math.pi, u_left, u_right)
    return np.tile(row, (n, 1)).astype(dtype)


def config_problem(name):
    """Problem parameters of the named workload (inputs only; no method logic).

    Returns a dict with the spectrum, kappa, macro grid size, band edges,
    patch grid per level and precision.
    """
    if name == "two_scale_cellular_fp64":          # 32^2 macro, 32^2 patches, 2 levels
        return dict(spectrum=cellular_two_scale(1.0, 1.0, 8), kappa=0.05, n_macro=32,
                    edges=[1.0, 8.0, 9.0], patch_n=[32, 32], precision="fp64",
                    cfl=0.2, T=1.0, sigma=0.5)
    if name == "three_level_cellular":            # 128^2 macro, 64^2 patches, 3 levels
        return dict(spectrum=cellular_hierarchy(3, 4), kappa=0.01, n_macro=128,
                    edges=[1.0, 4.0, 16.0, 64.0], patch_n=[64, 64, 64], precision="fp32",
                    cfl=0.2, T=1.0, sigma=0.5)
    if name == "continuous_spectrum":              # 256^2 macro, octave bands, 8 levels
        return dict(spectrum=continuous_spectrum(256), kappa=1e-3, n_macro=256,
                    edges=[1.0, 2.0, 4.0, 8.0, 16.0, 32.0, 64.0, 128.0, 257.0],
                    patch_n=None, precision="fp32", cfl=0.2, T=1.0, sigma=0.5)
    raise KeyError(name)


def mlp_init(d0, hidden, seed):
    """Seeded initial parameters of one surrogate member (FP32, layout
    W1[h][d0] b1 W2[h][h] b2 W3[h][h] b3 W4[3][h] b4): weights uniform in
    +-1/sqrt(fan_in), biases zero."""
    rng = np.random.default_rng(seed)
    parts = []
    for din, dout in [(d0, hidden), (hidden, hidden), (hidden, hidden), (hidden, 3)]:
        a = 1.0 / math.sqrt(din)
        parts.append(rng.uniform(-a, a, dout * din))
        parts.append(np.zeros(dout))
    return np.concatenate(parts).astype(np.float32)


def random_bases(P, kappa, seed, spread=1.5, cross=0.3):
    """Seeded symmetric positive definite base tensors around kappa:
    B11 = kappa e^a, B22 = kappa e^b (a, b uniform in [0, spread]),
    B12 = c sqrt(B11 B22) with c uniform in [-cross, cross]."""
    rng = np.random.default_rng(seed)
    a = kappa * np.exp(rng.uniform(0, spread, (P, 2)))
    c = rng.uniform(-cross, cross, P) * np.sqrt(a[:, 0] * a[:, 1])
    return np.stack([a[:, 0], c, a[:, 1]], 1)
