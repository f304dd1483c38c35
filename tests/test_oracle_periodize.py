"""Pins of the oracle's periodic-plus-smooth decomposition (the periodisation of
a band that is not periodic on its patch; Moisan 2011): u = p + s with the
periodic Laplacian of p equal to the Laplacian of u over in-patch neighbours
only, written out below with explicit differences; the seam jump of a
non-periodic band is gone from p; a constant field is its own periodic part."""
import numpy as np

import oracle


def _lap_per(f):
    return (np.roll(f, 1, 0) + np.roll(f, -1, 0) + np.roll(f, 1, 1) + np.roll(f, -1, 1) - 4 * f)


def _lap_int(f):
    n = f.shape[0]
    out = np.zeros_like(f)
    for b in range(n):
        for a in range(n):
            for db, da in ((1, 0), (-1, 0), (0, 1), (0, -1)):
                bb, aa = b + db, a + da
                if 0 <= bb < n and 0 <= aa < n:
                    out[b, a] += f[bb, aa] - f[b, a]
    return out


def test_defining_property_on_a_random_field():
    rng = np.random.default_rng(0)
    n = 12
    u = rng.standard_normal((n, n)) + np.linspace(0, 3, n)[None, :]
    p = oracle.periodic_smooth(u)
    np.testing.assert_allclose(_lap_per(p), _lap_int(u), atol=1e-12)
    assert abs(p.mean() - u.mean()) < 1e-13


def test_periodic_part_removes_the_seam_jump():
    # a band sampled on a patch that is not one of its periods has a jump across
    # the seam; the periodic part's seam differences are those of the interior
    n = 32
    x = 2 * np.pi * np.arange(n) / n
    u = np.sin(0.7 * x)[None, :] * np.cos(0.4 * x)[:, None]     # 0.7, 0.4 periods per patch
    p = oracle.periodic_smooth(u)
    seam_u = np.abs(u[:, 0] - u[:, -1]).max()
    seam_p = np.abs(p[:, 0] - p[:, -1]).max()
    step_p = np.abs(np.diff(p, axis=1)).max()
    assert seam_u > 5 * np.abs(np.diff(u, axis=1)).max()
    assert seam_p <= 1.5 * step_p


def test_constant_and_non_square_sizes():
    p = oracle.periodic_smooth(np.full((8, 8), 2.5))
    np.testing.assert_allclose(p, 2.5, atol=1e-14)
    # an odd size works the same way (the definition holds for any n)
    rng = np.random.default_rng(1)
    u = rng.standard_normal((9, 9))
    np.testing.assert_allclose(_lap_per(oracle.periodic_smooth(u)), _lap_int(u), atol=1e-12)
