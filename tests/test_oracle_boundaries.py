"""Pins of the oracle's boundary and incidence variants and of the solar-weighted totals:
a conductor (complex index) below the stack, oblique incidence (section "Photon
transport"), and Eq. 21 (section "Output")."""
import math

import numpy as np
import pytest


def _angle_form(ni, n2c, ci):
    """Reflectance from Snell's law with complex angles and the sine/tangent forms of
    the Fresnel amplitudes (a different route from the oracle's)."""
    ti = math.acos(ci)
    tt = np.arcsin(ni * np.sin(ti) / n2c + 0j)
    if abs(ti) < 1e-12:
        r = (ni - n2c) / (ni + n2c)
        return abs(r) ** 2
    rs = -np.sin(ti - tt) / np.sin(ti + tt)
    rp = np.tan(ti - tt) / np.tan(ti + tt)
    return 0.5 * (abs(rs) ** 2 + abs(rp) ** 2)


CONDUCTORS = [(1.0, 0.96, 6.69), (1.5, 1.2, 7.0), (1.0, 2.0, 0.1), (1.48, 0.05, 3.0),
              (1.33, 3.5, 0.01)]


@pytest.mark.parametrize("ni,n2,k2", CONDUCTORS)
def test_conductor_fresnel_vs_angle_form(orc, ni, n2, k2):
    for ci in (1.0, 0.9, 0.6, 0.3, 0.05):
        got = orc.fresnel_conductor(ni, n2, k2, ci)
        want = _angle_form(ni, complex(n2, k2), ci)
        assert abs(got - want) < 1e-12, (ci, got, want)
        f32 = orc.fresnel_conductor(ni, n2, k2, ci, fp32=True)
        assert abs(f32 - got) < 2e-6


def test_conductor_fresnel_limits(orc):
    for ni, n2, k2 in CONDUCTORS:
        normal = ((n2 - ni) ** 2 + k2 ** 2) / ((n2 + ni) ** 2 + k2 ** 2)
        assert abs(orc.fresnel_conductor(ni, n2, k2, 1.0) - normal) < 1e-14
        assert orc.fresnel_conductor(ni, n2, k2, 1e-9) > 1 - 1e-7   # grazing
    # vanishing k: the dielectric reflectance (no total internal reflection here)
    for ci in (1.0, 0.7, 0.2):
        R, _ = orc.fresnel(1.0, 1.6, ci)
        assert abs(orc.fresnel_conductor(1.0, 1.6, 1e-9, ci) - R) < 1e-8


def _slab(n=1.5, mu_a=0.4, d=1.0, N=200000, **kw):
    b = dict(n_stacks=1, n_wl=1, max_layers=1, mu_s=np.array([0.0]), mu_a=np.array([mu_a]),
             g=np.array([0.0]), n_layer=np.array([n]), thickness=np.array([d]),
             photons_per_item=N, seed=17)
    b.update(kw)
    return b


def _sigma_ok(count, N, p, k=4.5):
    s = math.sqrt(max(p * (1 - p), 1e-12) / N)
    return abs(count / N - p) <= k * s + 1e-12


@pytest.mark.parametrize("c0", [0.9, 0.6, 0.3])
def test_oblique_fresnel_slab_closed_form(orc, c0):
    mu_a, d, n = 0.4, 1.0, 1.5
    b = _slab(n, mu_a, d, cos_incidence=np.array([c0]))
    c = orc.mc_run(b, fp32=False)[0]
    r, ct = orc.fresnel(1.0, n, c0)
    tau = math.exp(-mu_a * d / ct)
    R = r + (1 - r) ** 2 * r * tau ** 2 / (1 - r * r * tau * tau)
    T = (1 - r) ** 2 * tau / (1 - r * r * tau * tau)
    N = b["photons_per_item"]
    assert c[:4].sum() == N
    assert _sigma_ok(c[0], N, R) and _sigma_ok(c[2], N, T)


def test_oblique_index_matched_beer_lambert_and_entry_tir(orc):
    b = _slab(1.0, 0.5, 1.0, cos_incidence=np.array([0.5]))
    c = orc.mc_run(b, fp32=False)[0]
    assert c[0] == 0
    assert _sigma_ok(c[2], b["photons_per_item"], math.exp(-0.5 / 0.5))
    # denser medium above, beyond the critical angle: every photon is reflected
    b = _slab(1.0, 0.5, 1.0, N=5000, cos_incidence=np.array([0.5]), n_above=np.array([1.5]))
    c = orc.mc_run(b, fp32=True)[0]
    assert c[0] == 5000 and c[4] == 0


def test_normal_incidence_stream_unchanged(orc):
    b = _slab(1.5, 0.1, 0.5, N=20000)
    b.update(mu_s=np.array([10.0]), g=np.array([0.7]))
    a = orc.mc_run(b, fp32=True)
    b2 = dict(b, cos_incidence=np.array([1.0]), k_below=np.array([0.0]))
    assert np.array_equal(a, orc.mc_run(b2, fp32=True))


@pytest.mark.parametrize("c0", [1.0, 0.5])
def test_conductor_below_closed_form(orc, c0):
    mu_a, d, n, nc, kc = 0.3, 1.0, 1.5, 1.2, 7.0
    b = _slab(n, mu_a, d, cos_incidence=np.array([c0]), n_below=np.array([nc]),
              k_below=np.array([kc]))
    c = orc.mc_run(b, fp32=False)[0]
    r, ct = orc.fresnel(1.0, n, c0)
    Rc = orc.fresnel_conductor(n, nc, kc, ct)
    tau = math.exp(-mu_a * d / ct)
    den = 1 - r * Rc * tau * tau
    R = r + (1 - r) ** 2 * Rc * tau * tau / den
    T = (1 - r) * tau * (1 - Rc) / den
    N = b["photons_per_item"]
    assert c[:4].sum() == N
    assert _sigma_ok(c[0], N, R) and _sigma_ok(c[2], N, T)


def _counts(fr, N=1000):
    """counts rows from fractions [rows, 3] (R, A, T) of N photons."""
    fr = np.asarray(fr, float)
    c = np.zeros((fr.shape[0], 6), np.int64)
    c[:, 0] = np.round(fr[:, 0] * N)
    c[:, 1] = np.round(fr[:, 1] * N)
    c[:, 2] = N - c[:, 0] - c[:, 1]
    return c


def test_solar_weighted_hand_example(orc):
    # R: 0.2, 0.4, 0.6 on lambda = 0.5, 1, 2 with G = 1, 2, 0.5:
    # num = 0.25 (0.2 + 0.8) + 0.5 (0.8 + 0.3) = 0.8, den = 0.25 * 3 + 0.5 * 2.5 = 2
    c = _counts([[0.2, 0.3, 0.5], [0.4, 0.1, 0.5], [0.6, 0.1, 0.3]])
    out = orc.solar_weighted(c, [0.5, 1.0, 2.0], [1.0, 2.0, 0.5], 1)
    assert abs(out[0, 0] - 0.4) < 1e-15
    # A: num = 0.25 (0.3 + 0.2) + 0.5 (0.2 + 0.05) = 0.25, / 2
    assert abs(out[0, 1] - 0.125) < 1e-15
    assert abs(out[0].sum() - 1.0) < 1e-15


def test_solar_weighted_constant_and_single_wavelength(orc):
    wl = np.linspace(0.3, 2.5, 50)
    G = np.exp(-((wl - 0.6) / 0.4) ** 2) + 0.01
    c = _counts(np.tile([[0.25, 0.5, 0.25]], (100, 1)))
    out = orc.solar_weighted(c, wl, G, 2)
    assert np.allclose(out, [[0.25, 0.5, 0.25]] * 2, rtol=0, atol=1e-15)
    one = orc.solar_weighted(_counts([[0.1, 0.2, 0.7]]), [0.5], [3.0], 1)
    assert np.allclose(one, [[0.1, 0.2, 0.7]], atol=1e-15)


def test_solar_weighted_trapezoid_converges(orc):
    """R(lambda) = lambda / 3 with G = 1 / lambda^2 on [0.3, 2.5]: the ratio of integrals
    is (ln(2.5/0.3) / 3) / (1/0.3 - 1/2.5); the trapezoidal error falls as h^2."""
    exact = (math.log(2.5 / 0.3) / 3) / (1 / 0.3 - 1 / 2.5)
    errs = []
    for n in (41, 81, 161):
        wl = np.linspace(0.3, 2.5, n)
        N = 10 ** 12
        fr = np.stack([wl / 3, np.zeros_like(wl), 1 - wl / 3], axis=1)
        c = _counts(fr, N)
        out = orc.solar_weighted(c, wl, 1 / wl ** 2, 1)
        errs.append(abs(out[0, 0] - exact))
    assert errs[0] / errs[1] > 3.5 and errs[1] / errs[2] > 3.5


SCATTERING = [
    # mu_s, mu_a, g, d, n, mu0, n_below, k_below
    (10.0, 0.1, 0.7, 0.5, 1.5, 0.5, 1.0, 0.0),
    (3.0, 1.0, 0.3, 1.0, 1.3, 0.8, 1.0, 0.0),
    (5.0, 0.5, 0.8, 0.5, 1.5, 1.0, 1.2, 7.0),
    (5.0, 0.5, 0.8, 0.5, 1.5, 0.4, 0.96, 6.69),
]


@pytest.mark.parametrize("case", SCATTERING)
def test_scattering_slab_oblique_and_conductor_vs_discrete_ordinates(orc, case):
    """Scattering slabs at oblique incidence and on a conductor against the
    discrete-ordinates solution of the transfer equation (an independent method)."""
    import rte_dom
    ms, ma, g, d, n, mu0, nb, kb = case
    ref = np.array(rte_dom.slab_rat(ms, ma, g, d, n, mu0=mu0, n_below=nb, k_below=kb))
    N = 400000
    b = _slab(n, ma, d, N=N, cos_incidence=np.array([mu0]), n_below=np.array([nb]))
    b.update(mu_s=np.array([ms]), g=np.array([g]), seed=23)
    if kb > 0:
        b["k_below"] = np.array([kb])
    c = orc.mc_run(b, fp32=True)[0]
    f = c[:3] / N
    sig = np.sqrt(ref * (1 - ref) / N)
    assert np.all(np.abs(f - ref) <= 4 * sig + 2e-4), (f, ref)
