"""Pins of the particle-size distribution (section "Scattering properties", last
paragraph) and of the library's host-side expansion (no GPU needed)."""
import math

import numpy as np
import pytest

from paper_2409_00165_gb300 import fos


def test_expansion_definition(orc):
    r, f = orc.size_distribution(0.5, 0.05, 0.002)
    assert len(r) == 101
    assert abs(f.sum() - 0.002) < 1e-17
    assert np.allclose(f, f[::-1], rtol=1e-14)                      # symmetric about D
    assert abs(f[0] / f[50] - math.exp(-4.5)) < 1e-14                 # ends at +-3 sigma
    assert abs(r[0] - 0.175) < 1e-15 and abs(r[-1] - 0.325) < 1e-15   # (D -+ 3 sigma)/2
    assert np.allclose(np.diff(r), 0.0015, rtol=1e-12)                # 6 sigma / 100 / 2
    r0, f0 = orc.size_distribution(0.5, 0.0, 0.002)
    assert list(r0) == [0.25] and list(f0) == [0.002]
    rt, ft = orc.size_distribution(0.1, 0.05, 0.002)                 # truncated at D > 0
    assert np.all(rt > 0) and len(rt) < 101 and abs(ft.sum() - 0.002) < 1e-17


def test_library_expansion_matches_definition(orc):
    for D, s, f in ((0.5, 0.05, 0.001), (0.5, 0.15, 0.001), (0.1, 0.05, 0.01), (1.0, 0.0, 0.1)):
        r1, f1 = orc.size_distribution(D, s, f)
        r2, f2 = fos.fos_size_distribution(D, s, f)
        assert len(r1) == len(r2)
        assert np.allclose(r1, r2, rtol=1e-15, atol=1e-17)
        assert np.allclose(f1, f2, rtol=1e-13, atol=1e-20)
    with pytest.raises(fos.FosError):
        fos.fos_size_distribution(-1.0, 0.1, 0.01)


def _medium(orc, dist, wl, m_p, m_h=1.33 + 0j):
    r, f = dist
    nm = np.array([[m_h] * len(wl)])
    n_p = np.array([[m_p] * len(wl)] * len(r))
    return orc.mie_properties(wl, nm, np.zeros(len(r), np.int32), n_p, r, f)


def test_narrow_distribution_tends_to_the_single_size(orc):
    wl = np.array([0.4, 0.8, 1.6])
    single = _medium(orc, orc.size_distribution(0.5, 0.0, 0.001), wl, 3.6 + 0.01j)
    narrow = _medium(orc, orc.size_distribution(0.5, 1e-6, 0.001), wl, 3.6 + 0.01j)
    for k in ("mu_s", "mu_a", "g"):
        assert np.allclose(narrow[k], single[k], rtol=1e-6)


def test_rayleigh_medium_scales_with_mean_cube(orc):
    """Small spheres scatter as r^6 per particle, so mu_s is proportional to the
    volume-weighted mean of r^3 over the distribution."""
    wl = np.array([5.0])
    dist = orc.size_distribution(0.02, 0.005, 0.001)
    got = _medium(orc, dist, wl, 1.6 + 0j)["mu_s"][0, 0]
    ref = _medium(orc, orc.size_distribution(0.02, 0.0, 0.001), wl, 1.6 + 0j)["mu_s"][0, 0]
    r, f = dist
    want = np.sum(f * r ** 3) / (0.001 * 0.01 ** 3)
    assert abs(got / ref / want - 1) < 2e-4
