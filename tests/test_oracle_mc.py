"""Pins of the oracle's Monte Carlo photon walk (section "Photon transport").

Closed forms (Beer-Lambert, Fresnel slab, opaque reflector, incoherent adding of
non-scattering layers), invariants (conservation, mu_a = 0 -> A = 0, sharding) and
an independent deterministic RTE solution (discrete ordinates) for scattering slabs.
"""
import math
import os

import numpy as np
import pytest

from rte_dom import fresnel_angle_form, slab_rat
from paper_2409_00165_gb300 import workloads as W

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _batch(mu_s, mu_a, g, n, d, N, n_above=1.0, n_below=1.0, sub=None, seed=1, **kw):
    L = len(mu_s)
    b = dict(n_stacks=1, n_wl=1, max_layers=L, n_layers=np.array([L], np.int32),
             mu_s=np.array(mu_s, float), mu_a=np.array(mu_a, float), g=np.array(g, float),
             n_layer=np.array(n, float), thickness=np.array(d, float),
             n_above=np.array([n_above]), n_below=np.array([n_below]),
             photons_per_item=int(N), seed=seed)
    if sub is not None:
        b["substrate_R"] = np.array([sub])
    b.update(kw)
    return b


def _within(frac, p, N, nsig=4.0, extra=0.0):
    sig = math.sqrt(max(p * (1 - p), 1e-12) / N)
    return abs(frac - p) <= nsig * sig + extra


# ---------------------------------------------------------------- components
def test_fresnel_against_angle_form(orc):
    for ni, nt in [(1.0, 1.5), (1.5, 1.0), (1.33, 2.1), (2.4, 1.48)]:
        for ci in np.linspace(0.02, 1.0, 50):
            R, ct = orc.fresnel(ni, nt, ci)
            ref = fresnel_angle_form(ni, nt, np.array([ci]))[0]
            assert abs(R - ref) <= 1e-12 * max(1.0, ref) + 1e-14
    # normal incidence closed form
    R, ct = orc.fresnel(1.0, 1.5, 1.0)
    assert abs(R - 0.04) < 1e-15 and ct == 1.0
    # total internal reflection beyond the critical angle, R -> 1 at grazing
    mu_c = math.sqrt(1 - (1 / 1.5) ** 2)
    assert orc.fresnel(1.5, 1.0, mu_c * 0.999)[0] == 1.0
    assert orc.fresnel(1.0, 1.5, 1e-6)[0] > 0.9999
    # Brewster angle: p reflectance vanishes, so R = R_s / 2
    tb = math.atan(1.5)
    R, _ = orc.fresnel(1.0, 1.5, math.cos(tb))
    tt = math.asin(math.sin(tb) / 1.5)
    rs = (math.sin(tb - tt) / math.sin(tb + tt)) ** 2
    assert abs(R - rs / 2) < 1e-14


def _hg_cdf(g, mu):
    return (1 - g * g) / (2 * g) * ((1 + g * g - 2 * g * mu) ** -0.5 - 1 / (1 + g))


@pytest.mark.parametrize("g", [-0.9, -0.3, 0.2, 0.7, 0.95])
def test_hg_inverse_cdf(orc, g):
    """The sampled cosine is the inverse of the HG cumulative distribution."""
    u = (np.arange(2000) + 0.5) / 2000
    c = np.array([orc.hg_cos(g, x) for x in u])
    assert np.max(np.abs(_hg_cdf(g, c) - u)) < 1e-12
    # midpoint rule over u: mean cosine = g
    uu = (np.arange(200000) + 0.5) / 200000
    cc = np.array([orc.hg_cos(g, x) for x in uu[::50]])
    assert abs(np.mean(cc) - g) < 5e-4


def test_hg_fp32_histogram(orc):
    """FP32 sampler: mean cosine within 4 sigma and chi-square vs the HG pdf."""
    g = 0.7
    rng = np.random.default_rng(5)
    u = (2 * rng.integers(0, 2 ** 23, size=100000) + 1) * 2.0 ** -24
    c = np.array([orc.hg_cos(g, float(x), fp32=True) for x in u])
    n = c.size
    m2 = (1 + 2 * g * g) / 3  # <cos^2> of HG
    sig = math.sqrt((m2 - g * g) / n)
    assert abs(c.mean() - g) < 4 * sig
    edges = np.linspace(-1, 1, 101)
    h, _ = np.histogram(c, bins=edges)
    p = np.diff(_hg_cdf(g, edges))
    e = n * p
    ok = e > 5
    chi2 = np.sum((h[ok] - e[ok]) ** 2 / e[ok])
    dof = ok.sum() - 1
    assert chi2 < dof + 5 * math.sqrt(2 * dof)
    # isotropic special case
    assert orc.hg_cos(0.0, 0.25) == -0.5


# ---------------------------------------------------------------- closed forms
@pytest.mark.parametrize("fp32", [True, False])
def test_beer_lambert_index_matched(orc, fp32):
    N = 200000
    for n in (1.0, 1.5):
        c = orc.mc_run(_batch([0.0], [0.1], [0.0], [n], [0.5], N, n, n), fp32=fp32)[0]
        assert c[0] == 0                       # no interface, no scattering: R = 0
        assert c[0] + c[1] + c[2] + c[3] == N
        assert _within(c[2] / N, math.exp(-0.05), N)


def test_fresnel_slab_closed_form(orc):
    vals = {}
    with open(os.path.join(GOLDEN, "fresnel_slab.txt")) as fh:
        for line in fh:
            if line.strip() and not line.startswith("#"):
                k, v = line.split()
                vals[k] = float(v)
    r, tau = 0.04, math.exp(-0.05)
    R = r + (1 - r) ** 2 * r * tau ** 2 / (1 - r * r * tau * tau)
    T = (1 - r) ** 2 * tau / (1 - r * r * tau * tau)
    assert abs(R - vals["R"]) < 1e-6 and abs(T - vals["T"]) < 1e-6
    assert abs(1 - R - T - vals["A"]) < 1e-6
    N = 400000
    for fp32 in (True, False):
        c = orc.mc_run(_batch([0.0], [0.1], [0.0], [1.5], [0.5], N), fp32=fp32)[0]
        assert _within(c[0] / N, R, N) and _within(c[2] / N, T, N)
        assert _within(c[1] / N, 1 - R - T, N)


def _adding(elems):
    """Incoherent adding of elements (Rf, Tf, Rb, Tb), top first."""
    Rf, Tf, Rb, Tb = elems[0]
    for (R2f, T2f, R2b, T2b) in elems[1:]:
        den = 1 - Rb * R2f
        nRf = Rf + Tf * Tb * R2f / den
        nTf = Tf * T2f / den
        nRb = R2b + T2b * T2f * Rb / den
        nTb = T2b * Tb / den
        Rf, Tf, Rb, Tb = nRf, nTf, nRb, nTb
    return Rf, Tf


def _iface(na, nb):
    r = ((na - nb) / (na + nb)) ** 2
    return (r, 1 - r, r, 1 - r)


def _layer(mua, d):
    t = math.exp(-mua * d)
    return (0.0, t, 0.0, t)


def test_two_layer_non_scattering_adding(orc):
    n1, n2 = 1.5, 2.0
    ma, d = [0.3, 0.8], [0.4, 0.25]
    R, T = _adding([_iface(1.0, n1), _layer(ma[0], d[0]), _iface(n1, n2),
                    _layer(ma[1], d[1]), _iface(n2, 1.2)])
    N = 300000
    c = orc.mc_run(_batch([0, 0], ma, [0, 0], [n1, n2], d, N, 1.0, 1.2), fp32=True)[0]
    assert _within(c[0] / N, R, N) and _within(c[2] / N, T, N)
    assert c[0] + c[1] + c[2] == N


def test_opaque_reflector_closed_form(orc):
    r = 0.04
    tau = math.exp(-0.3 * 0.5)
    Rs = 0.35
    R = r + (1 - r) ** 2 * Rs * tau ** 2 / (1 - r * Rs * tau ** 2)
    T = (1 - r) * tau * (1 - Rs) / (1 - r * Rs * tau ** 2)
    N = 300000
    c = orc.mc_run(_batch([0.0], [0.3], [0.0], [1.5], [0.5], N, sub=Rs), fp32=True)[0]
    assert _within(c[0] / N, R, N) and _within(c[2] / N, T, N)
    # adding method agrees with the closed form
    Ra, Ta = _adding([_iface(1.0, 1.5), _layer(0.3, 0.5), (Rs, 1 - Rs, 0.0, 0.0)])
    assert abs(Ra - R) < 1e-14 and abs(Ta - T) < 1e-14


# ---------------------------------------------------------------- invariants
def test_conservation_and_no_absorption(orc):
    N = 20000
    b = _batch([5.0, 2.0], [0.0, 0.0], [0.8, -0.2], [1.4, 1.7], [0.3, 0.6], N, 1.0, 1.3)
    c = orc.mc_run(b, fp32=True)[0]
    assert c[1] == 0
    assert c[0] + c[1] + c[2] + c[3] == N
    assert c[3] == 0


def test_runaway_cap(orc):
    N = 2000
    b = _batch([50.0], [0.0], [0.9], [1.5], [2.0], N, max_events=30)
    c = orc.mc_run(b, fp32=True)[0]
    assert c[3] > 0
    assert c[0] + c[1] + c[2] + c[3] == N
    # no photon has more than max_events events
    assert c[4] + c[5] <= 30 * N


def test_photon_range_sharding_is_exact(orc):
    """Results depend only on photon ids: split ranges sum to the whole run."""
    N = 6000
    base = _batch([10.0], [0.1], [0.7], [1.5], [0.5], N)
    full = orc.mc_run(base, fp32=True)[0]
    parts = np.zeros(6, np.int64)
    for first, cnt in [(0, 2500), (2500, 1000), (3500, 2500)]:
        b = dict(base)
        b["photons_per_item"] = cnt
        b["photon_first"] = np.array([first], np.int64)
        parts += orc.mc_run(b, fp32=True)[0]
    assert np.array_equal(full, parts)


def test_item_list_selects_rows(orc):
    b = _batch([10.0], [0.1], [0.7], [1.5], [0.5], 3000)
    b.update(n_wl=3, mu_s=np.array([10.0, 4.0, 1.0]), mu_a=np.array([0.1, 0.2, 0.3]),
             g=np.array([0.7, 0.5, 0.0]), n_layer=np.array([1.5, 1.4, 1.3]),
             n_above=np.ones(3), n_below=np.ones(3))
    all_rows = orc.mc_run(b, fp32=True)
    b2 = dict(b)
    b2["item_list"] = np.array([2, 0], np.int32)
    sel = orc.mc_run(b2, fp32=True)
    assert np.array_equal(sel[0], all_rows[2]) and np.array_equal(sel[1], all_rows[0])


def test_identical_sublayers_match_single_layer(orc):
    N = 200000
    one = orc.mc_run(_batch([4.0], [0.5], [0.6], [1.4], [0.6], N), fp32=False)[0]
    two = orc.mc_run(_batch([4.0, 4.0], [0.5, 0.5], [0.6, 0.6], [1.4, 1.4], [0.3, 0.3], N,
                            seed=99), fp32=False)[0]
    for k in range(3):
        p = one[k] / N
        assert abs(two[k] / N - p) <= 5 * math.sqrt(2 * p * (1 - p) / N)


def test_fp32_mirror_agrees_with_fp64(orc):
    N = 100000
    b = W.single_slab(N)
    c32 = orc.mc_run(b, fp32=True)[0]
    c64 = orc.mc_run(b, fp32=False)[0]
    for k in range(3):
        assert abs(c32[k] - c64[k]) / N <= 1e-3
    assert c32[:4].sum() == N and c64[:4].sum() == N


# ---------------------------------------------------------------- scattering slabs vs RTE
@pytest.mark.parametrize("case", [
    # mu_s, mu_a, g, d, n_in, n_above, n_below, photons
    (10.0, 0.1, 0.7, 0.5, 1.5, 1.0, 1.0, 1000000),     # the single-slab workload
    (3.0, 0.3, -0.5, 1.0, 1.33, 1.33, 1.33, 400000),   # back-scattering, index matched
    (4.0, 1.0, 0.0, 0.8, 1.4, 1.0, 1.6, 400000),       # isotropic, unequal boundaries
])
def test_scattering_slab_vs_discrete_ordinates(orc, case):
    ms, ma, g, d, n, na, nb, N = case
    ref = slab_rat(ms, ma, g, d, n, na, nb, n_half=96)
    b = _batch([ms], [ma], [g], [n], [d], N, na, nb, seed=11)
    for fp32 in (False, True):
        c = orc.mc_run(b, fp32=fp32)[0]
        for k in range(3):
            # 4 sigma binomial plus 2e-4 for the quadrature of the deterministic solver
            assert _within(c[k] / N, ref[k], N, 4.0, 2e-4), (fp32, k, c[k] / N, ref[k])
