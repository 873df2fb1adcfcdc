"""Pins of the oracle's Mie theory (Eqs. 1-5, 10-12, 15) and effective medium (13-20)."""
import math

import mpmath as mp
import numpy as np
import pytest
from scipy import special

from paper_2409_00165_gb300 import workloads as W


# ---------------------------------------------------------------- a_n, b_n by brute force
def _mp_coeffs(wl, n_p, n_m, r, N, dps=40):
    """a_n, b_n from Eqs. 2-5 with psi_n = sqrt(pi z/2) J_{n+1/2}(z) and
    xi_n = sqrt(pi z/2) H^(1)_{n+1/2}(z) evaluated by mpmath; derivatives from the
    identity f_n' = f_{n-1} - n f_n / z of Riccati-Bessel functions."""
    with mp.workdps(dps):
        n_p, n_m = mp.mpc(n_p), mp.mpc(n_m)
        x = 2 * mp.pi * r * n_m / wl
        y = 2 * mp.pi * r * n_p / wl
        half = mp.mpf(1) / 2

        def psi(n, z):
            return mp.sqrt(mp.pi * z / 2) * mp.besselj(n + half, z)

        def xi(n, z):
            return mp.sqrt(mp.pi * z / 2) * (mp.besselj(n + half, z)
                                             + 1j * mp.bessely(n + half, z))
        out = []
        px_prev, py_prev, xx_prev = psi(0, x), psi(0, y), xi(0, x)
        for n in range(1, N + 1):
            px, py, xx = psi(n, x), psi(n, y), xi(n, x)
            Ax = (px_prev - n * px / x) / px
            Ay = (py_prev - n * py / y) / py
            Bx = (xx_prev - n * xx / x) / xx
            ratio = px / xx
            a = ratio * (n_m * Ay - n_p * Ax) / (n_m * Ay - n_p * Bx)
            b = ratio * (n_p * Ay - n_m * Ax) / (n_p * Ay - n_m * Bx)
            out.append((complex(a), complex(b)))
            px_prev, py_prev, xx_prev = px, py, xx
        return np.array(out)


MIE_POINTS = [
    # wl, n_p, n_m, r   (covers the workloads: visible/UV/IR, r 0.05..1 um)
    (0.5, 2.7 + 1e-4j, 1.48 + 5e-6j, 0.2),
    (0.3, 3.0556 + 0.5j, 1.48 + 3e-6j, 1.0),      # |y| ~ 64, Im y ~ 10.5
    (0.35, 2.908 + 0.5j, 1.48 + 3.5e-6j, 0.6),
    (2.5, 2.508 + 1e-4j, 1.48 + 2.5e-5j, 0.05),   # Rayleigh-like
    (1.2, 2.535 + 1e-4j, 1.48 + 1.2e-5j, 0.75),
    (0.55, 1.33 + 1e-8j, 1.0 + 0j, 1.0),          # water droplet in air
    (0.8, 1.5 + 0.02j, 1.33 + 1e-7j, 0.4),
]


@pytest.mark.parametrize("pt", MIE_POINTS)
def test_mie_coefficients_vs_mpmath(orc, pt):
    wl, n_p, n_m, r = pt
    o = orc.mie_sphere(wl, n_p, n_m, r, with_coeffs=True)
    N = o["n_max"] + 1
    ref = _mp_coeffs(wl, n_p, n_m, r, N)
    scale_a = np.max(np.abs(ref[:, 0]))
    scale_b = np.max(np.abs(ref[:, 1]))
    # relative to each coefficient where it matters, else to the largest one
    ea = np.abs(o["a"] - ref[:, 0]) / np.maximum(np.abs(ref[:, 0]), 1e-6 * scale_a)
    eb = np.abs(o["b"] - ref[:, 1]) / np.maximum(np.abs(ref[:, 1]), 1e-6 * scale_b)
    assert ea.max() < 1e-11 and eb.max() < 1e-11


def test_nmax_formula(orc):
    o = orc.mie_sphere(0.3, 3.0556 + 0.5j, 1.48, 1.0)
    y = abs(2 * math.pi * 1.0 * (3.0556 + 0.5j) / 0.3)
    assert o["n_max"] == math.ceil(2 + y + 4.3 * y ** (1 / 3))


def test_log_derivative_vs_scipy(orc):
    for n in (1, 3, 10, 25):
        for z in (0.7 + 0.0j, 5.3 + 0.01j, 12.0 + 2.0j, 3.0 + 0.5j):
            jn = special.spherical_jn(n, z)
            jd = special.spherical_jn(n, z, derivative=True)
            ref = (jn + z * jd) / (z * jn)          # psi'/psi with psi = z j_n
            got = orc.log_deriv_psi(n, z)
            assert abs(got - ref) <= 1e-10 * abs(ref)


# ---------------------------------------------------------------- limits and invariants
def test_rayleigh_limit(orc):
    m = 1.6 + 0.05j
    wl, r = 1.0, 2e-4
    x = 2 * math.pi * r / wl
    o = orc.mie_sphere(wl, m, 1.0, r)
    K = (m * m - 1) / (m * m + 2)
    q_sca = 8 / 3 * x ** 4 * abs(K) ** 2
    q_abs = 4 * x * K.imag
    assert abs(o["q_sca"] / q_sca - 1) < 1e-5
    assert abs((o["q_ext"] - o["q_sca"]) / q_abs - 1) < 1e-5
    assert abs(o["g"]) < 1e-5


@pytest.mark.parametrize("m,x", [(1.33, 1.0), (2.0, 5.0), (1.5, 30.0), (2.6, 12.0)])
def test_energy_conservation_non_absorbing(orc, m, x):
    """Optical theorem: a non-absorbing sphere in a non-absorbing host has
    Q_ext = Q_sca."""
    wl = 1.0
    r = x * wl / (2 * math.pi)
    o = orc.mie_sphere(wl, m + 0j, 1.0, r)
    assert abs(o["q_ext"] - o["q_sca"]) <= 1e-11 * o["q_ext"]


def _pi_tau(nmax, mu):
    """Angular functions pi_n, tau_n (Bohren & Huffman recurrences)."""
    pi = np.zeros((nmax + 1, mu.size))
    tau = np.zeros((nmax + 1, mu.size))
    pi[1] = 1.0
    if nmax >= 2:
        pi[2] = 3 * mu
    for n in range(3, nmax + 1):
        pi[n] = (2 * n - 1) / (n - 1) * mu * pi[n - 1] - n / (n - 1) * pi[n - 2]
    for n in range(1, nmax + 1):
        tau[n] = n * mu * pi[n] - (n + 1) * pi[n - 1] if n > 1 else mu * pi[1]
    return pi, tau


@pytest.mark.parametrize("pt", [(0.5, 2.7 + 1e-4j, 0.2), (0.55, 1.33 + 1e-8j, 1.0),
                                (0.8, 1.5 + 0.02j, 0.4), (0.3, 3.0556 + 0.5j, 1.0)])
def test_asymmetry_from_phase_function(orc, pt):
    """g of Eq. 15 and Q_sca of Eq. 12 equal the moments of the scattered intensity
    |S1|^2 + |S2|^2 integrated over angle (non-absorbing host)."""
    wl, m, r = pt
    o = orc.mie_sphere(wl, m, 1.0, r, with_coeffs=True)
    nmax = o["n_max"]
    a, b = o["a"][:nmax], o["b"][:nmax]
    mu, w = np.polynomial.legendre.leggauss(2 * nmax + 40)
    pi, tau = _pi_tau(nmax, mu)
    n = np.arange(1, nmax + 1)[:, None]
    c = (2 * n + 1) / (n * (n + 1))
    S1 = np.sum(c * (a[:, None] * pi[1:] + b[:, None] * tau[1:]), axis=0)
    S2 = np.sum(c * (a[:, None] * tau[1:] + b[:, None] * pi[1:]), axis=0)
    I = np.abs(S1) ** 2 + np.abs(S2) ** 2
    x = 2 * math.pi * r / wl
    q_sca = np.sum(w * I) / (x * x)            # (1/x^2) int (|S1|^2+|S2|^2) dmu
    g = np.sum(w * I * mu) / np.sum(w * I)
    assert abs(q_sca / o["q_sca"] - 1) < 1e-10
    assert abs(g - o["g"]) < 1e-10


def test_large_sphere_extinction_limit(orc):
    """Large spheres: Q_ext -> 2 with the edge term 1.9924 x^(-2/3) (Nussenzveig and
    Wiscombe 1980) once internal absorption damps the interference ripple."""
    for x in (400.0, 753.9822368615503, 1500.0):      # the middle one is 240 pi
        r = x * 0.5 / (2 * math.pi)
        o = orc.mie_sphere(0.5, 1.5 + 0.01j, 1.0, r)
        assert abs((o["q_ext"] - 2.0) * x ** (2 / 3) - 1.9924) < 0.05


def test_gamma_geometric_term(orc):
    # series branch continues the closed form of Eq. 10 smoothly, gamma(0) = 1
    assert abs(orc.gamma_term(0.0) - 1.0) < 1e-15
    for a in (0.5, 0.8, 1.5, 4.0):
        closed = 2 * (1 + (a - 1) * math.exp(a)) / (a * a)
        assert abs(orc.gamma_term(a) - closed) < 1e-14 * closed
    with mp.workdps(50):
        for a in (1e-8, 1e-4, 0.05, 0.3, 0.4999):
            mpv = mp.mpf(2) * (1 + (mp.mpf(a) - 1) * mp.exp(mp.mpf(a))) / mp.mpf(a) ** 2
            assert abs(orc.gamma_term(a) - float(mpv)) < 2e-15 * float(mpv)


def test_absorbing_host_reduces_to_textbook(orc):
    # k_m -> 0 is continuous: the absorbing-host result approaches k_m = 0.
    a = orc.mie_sphere(0.6, 2.6 + 1e-4j, 1.48 + 0j, 0.3)
    b = orc.mie_sphere(0.6, 2.6 + 1e-4j, 1.48 + 1e-12j, 0.3)
    for k in ("q_ext", "q_sca", "g"):
        assert abs(a[k] - b[k]) < 1e-9 * abs(a[k])


# ---------------------------------------------------------------- effective medium
def test_effective_medium_arithmetic(orc):
    wl = np.array([0.5, 1.0, 2.0])
    nm = np.array([[1.48 + 1e-5j, 1.48 + 2e-5j, 1.48 + 4e-5j]] * 4)
    n_p = np.array([[2.6 + 1e-4j] * 3] * 5)
    # group 0: f = 0.05 (no correction); group 1: f = 0.10 (C = 1.1425);
    # group 2: two species of the same particle, 0.04 + 0.06; group 3: no particles
    sg = [0, 1, 2, 2, 2]
    rad = [0.2, 0.2, 0.2, 0.2, 0.3]
    vf = [0.05, 0.10, 0.04, 0.06, 0.0]
    o = orc.mie_properties(wl, nm, sg, n_p, rad, vf)
    mat = 4 * math.pi * nm.imag / wl[None, :]
    # matrix absorption alone (Eq. 20 with no particles): mu_a = 4 pi k / lambda
    assert np.allclose(o["mu_a"][3], mat[3], rtol=1e-14) and np.all(o["mu_s"][3] == 0)
    # Eq. 13 with one species: mu_s = 1.5 q f / (2 r)
    q = o["q_sca"][0]
    assert np.allclose(o["mu_s"][0], 1.5 * q * 0.05 / 0.4, rtol=1e-14)
    # crossing 0.08 multiplies by C(0.1) = 1 + 0.15 - 0.0075 = 1.1425
    assert np.allclose(o["mu_s"][1] / o["mu_s"][0], 2 * 1.1425, rtol=1e-13)
    pa0 = o["mu_a"][0] - mat[0] * 0.95
    pa1 = o["mu_a"][1] - mat[1] * 0.90
    assert np.allclose(pa1 / pa0, 2 * 1.1425, rtol=1e-9)
    # additivity: two species 0.04 + 0.06 of one particle = one species of 0.10
    assert np.allclose(o["mu_s"][2], o["mu_s"][1], rtol=1e-13)
    assert np.allclose(o["g"][2], o["g"][1], rtol=1e-13)
    # g of the medium is the g of its only particle size
    assert np.allclose(o["g"][0], o["g_sp"][0], rtol=1e-14)


def test_dependent_scattering_factor_at_0_3(orc):
    wl = np.array([0.7])
    nm = np.array([[1.48 + 0j], [1.48 + 0j]])
    n_p = np.array([[2.6 + 0j], [2.6 + 0j]])
    o = orc.mie_properties(wl, nm, [0, 1], n_p, [0.25, 0.25], [0.03, 0.3])
    # C(0.3) = 1 + 0.45 - 0.0675 = 1.3825
    assert abs(o["mu_s"][1, 0] / o["mu_s"][0, 0] - 10 * 1.3825) < 1e-12


def test_workload_materials_are_finite(orc):
    m = W.paint_layer(n_wl=16)
    o = orc.mie_properties(m["wl"], m["nm"], m["species_group"], m["n_p"], m["radius"],
                           m["vol_frac"])
    for k in ("mu_s", "mu_a", "g"):
        assert np.all(np.isfinite(o[k]))
    assert np.all(o["mu_s"] > 0) and np.all(o["mu_a"] > 0)
    assert np.all((o["g"] > 0) & (o["g"] < 1))
