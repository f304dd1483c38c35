"""Pins of the oracle's patch-resolution rule for uneven patch sizes.

The rule (the reading of the paper's resolution requirement for local
problems: at least 10 points per wavelength, as the Sec. 4 reference solutions
use, and a cell Peclet number of at most 2 with the molecular diffusivity) is

    n = clamp(pow2ceil(max(10 kmax L / 2pi, L vmax / (2 kappa))), n_min, n_max)

with L = 2 pi / m_l the level's patch side, kmax = max(|k1|, |k2|) over the
level's diagonal modes and vmax the largest speed |v| of the band's velocity
on the patch's reference nodes.  Each case below has kmax and vmax known by
hand, and sits on one side of a power of two so that a wrong factor (10 points
per wavelength, the patch side, the 1/2 of the Peclet bound, |v| against
|v1| + |v2| or |v1| alone) moves n to another power of two.
"""
import math

import numpy as np
import pytest

from inputs import flows
import oracle

EDGES = [1.0, 4.0, 16.0, 64.0]     # level l has m_l = 1, 4, 16 and L_l = 2 pi / m_l


def _ref_nodes(i, n_macro, m, nref=32):
    """Lattice indices of the reference nodes of macro node i: the lattice has
    Nr = nref * m points and the patch centre is the node nearest to
    i * Nr / n_macro (here an exact node), node a at centre - nref/2 + a."""
    Nr = nref * m
    c = i * Nr // n_macro
    assert c * n_macro == i * Nr
    return (c - nref // 2 + np.arange(nref)), Nr


def _diag_vmax(terms, node, n_macro, m):
    """max over the reference nodes of |v| for psi = sum_q A_q sin(k_q (x1 + x2)):
    v = (-d2 psi, d1 psi) = s(x) (-1, 1) with s = sum_q A_q k_q cos(k_q (x1 + x2)),
    so |v| = sqrt(2) |s|."""
    ga, Nr = _ref_nodes(node[0], n_macro, m)
    gb, _ = _ref_nodes(node[1], n_macro, m)
    x = 2 * math.pi * (ga[None, :] + gb[:, None]) / Nr
    s = sum(A * k * np.cos(k * x) for A, k in terms)
    return math.sqrt(2.0) * np.abs(s).max()


def _diag(terms):
    return flows.combine(*[flows.shear_diag(A, k) for A, k in terms])


@pytest.mark.parametrize("k,want", [(12, 32), (13, 64)])
def test_resolution_branch(k, want):
    # level 2 (m = 4, L = pi/2): 10 k L / 2 pi = 10 k / 4 = 30 -> 32, 32.5 -> 64;
    # the Peclet term is ~1.4 (A = 1e-3, kappa = 1e-2)
    spec = _diag([(1e-3, k)])
    n, vmax = oracle.patch_n_rule(spec, EDGES, 2, (0, 0), 4, 1e-2, n_min=8, n_max=256)
    assert vmax == pytest.approx(math.sqrt(2) * 1e-3 * k, rel=1e-12)
    assert n == want


@pytest.mark.parametrize("pe,want", [(100.0, 128), (70.0, 128), (120.0, 128), (60.0, 64)])
def test_peclet_branch(pe, want):
    # level 1 (m = 1, L = 2 pi), mode k = 2 on the diagonal: 10 k L / 2 pi = 20;
    # vmax = sqrt(2) A k exactly (a reference node has cos(k(x1 + x2)) = 1), so
    # L vmax / (2 kappa) = 2 pi sqrt(2) A k / (2 kappa) = pe for the amplitude below.
    # pe = 100: |v1| + |v2| would give 141 -> 256, and L vmax / kappa 200 -> 256;
    # pe = 70: |v1| alone would give 49.5 -> 64.
    kappa, k = 1e-2, 2
    A = pe * 2 * kappa / (2 * math.pi * math.sqrt(2) * k)
    spec = _diag([(A, k)])
    n, vmax = oracle.patch_n_rule(spec, EDGES, 1, (1, 2), 4, kappa, n_min=8, n_max=256)
    assert vmax == pytest.approx(math.sqrt(2) * A * k, rel=1e-12)
    assert n == want


def test_two_mode_band_and_other_parts_ignored():
    # level 2 holds k = 5 and k = 13 on the diagonal: kmax = 13 -> 10*13/4 = 32.5 -> 64,
    # vmax from both modes at once.  Modes of other parts do not count: an
    # off-diagonal mode of level 1 ((2, 40): |k1| in level 1, |k2| in level 3) and
    # a diagonal mode of level 3 ((20, 20)), both with large amplitudes.
    terms = [(3e-3, 5), (1e-3, 13)]
    kappa = 1e-2
    spec = flows.combine(_diag(terms), flows.shear_diag(5.0, 20),
                         flows._from_dict({(2, 40): 2.0 - 1.0j, (-2, -40): 2.0 + 1.0j}))
    lev, kind = oracle.band_of(spec, EDGES)
    k1 = spec.k1
    assert all(lev[t] == 1 and kind[t] != 0 for t in range(len(k1)) if abs(k1[t]) == 2)
    for node in [(0, 0), (3, 1), (2, 2)]:
        n, vmax = oracle.patch_n_rule(spec, EDGES, 2, node, 4, kappa, n_min=8, n_max=256)
        assert vmax == pytest.approx(_diag_vmax(terms, node, 4, 4), rel=1e-12)
        assert n == 64


@pytest.mark.parametrize("n_min,n_max,A,want", [
    (32, 256, 1e-4, 32),      # need 10*20/16 = 12.5 -> 16, raised to n_min
    (8, 256, 1e-4, 16),       # the same case without the floor
    (32, 256, 50.0, 256),     # Peclet term ~ 1e4: capped at n_max
    (32, 128, 50.0, 128),
])
def test_clamps(n_min, n_max, A, want):
    # level 3 (m = 16, L = pi/8), mode k = 20 on the diagonal
    spec = _diag([(A, 20)])
    n, _ = oracle.patch_n_rule(spec, EDGES, 3, (1, 1), 4, 1e-2, n_min=n_min, n_max=n_max)
    assert n == want
