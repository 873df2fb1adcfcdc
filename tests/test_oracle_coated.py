"""Pins of the oracle's core-shell Mie theory (supplement Eqs. S1-S9)."""
import math

import mpmath as mp
import numpy as np
import pytest


def _mp_coated(wl, n_c, n_s, n_m, a, b, N, dps=40):
    """a_n, b_n from S1-S9 with psi_n = sqrt(pi z/2) J_{n+1/2}(z),
    chi_n = sqrt(pi z/2) Y_{n+1/2}(z), xi_n = psi_n + i chi_n (mpmath, 40 digits);
    derivatives from f_n' = f_{n-1} - n f_n / z."""
    with mp.workdps(dps):
        n_c, n_s, n_m = mp.mpc(n_c), mp.mpc(n_s), mp.mpc(n_m)
        m1, m2 = n_c / n_m, n_s / n_m
        k = 2 * mp.pi / wl
        x, y = k * a * n_m, k * b * n_m
        half = mp.mpf(1) / 2

        def psi(n, z):
            return mp.sqrt(mp.pi * z / 2) * mp.besselj(n + half, z)

        def chi(n, z):
            return mp.sqrt(mp.pi * z / 2) * mp.bessely(n + half, z)

        def d(f, n, z):
            return f(n - 1, z) - n * f(n, z) / z

        out = []
        for n in range(1, N + 1):
            xi = lambda nn, z: psi(nn, z) + 1j * chi(nn, z)
            An = ((m2 * psi(n, m2 * x) * d(psi, n, m1 * x) - m1 * d(psi, n, m2 * x) * psi(n, m1 * x))
                  / (m2 * chi(n, m2 * x) * d(psi, n, m1 * x) - m1 * d(chi, n, m2 * x) * psi(n, m1 * x)))
            Bn = ((m2 * psi(n, m1 * x) * d(psi, n, m2 * x) - m1 * psi(n, m2 * x) * d(psi, n, m1 * x))
                  / (m2 * d(chi, n, m2 * x) * psi(n, m1 * x) - m1 * d(psi, n, m1 * x) * chi(n, m2 * x)))
            Ua = d(psi, n, m2 * y) - An * d(chi, n, m2 * y)
            Va = psi(n, m2 * y) - An * chi(n, m2 * y)
            Ub = d(psi, n, m2 * y) - Bn * d(chi, n, m2 * y)
            Vb = psi(n, m2 * y) - Bn * chi(n, m2 * y)
            an = (psi(n, y) * Ua - m2 * d(psi, n, y) * Va) / (xi(n, y) * Ua - m2 * d(xi, n, y) * Va)
            bn = (m2 * psi(n, y) * Ub - d(psi, n, y) * Vb) / (m2 * xi(n, y) * Ub - d(xi, n, y) * Vb)
            out.append((complex(an), complex(bn)))
        return np.array(out)


POINTS = [
    # wl, n_core, n_shell, n_m, a, b
    (0.8, 1.0 + 0j, 1.45 + 1e-4j, 1.0 + 0j, 0.25, 0.35),     # hollow silica in air
    (0.5, 2.5 + 0.1j, 1.45 + 0j, 1.33 + 1e-7j, 0.1, 0.3),    # absorbing core, silica shell
    (1.5, 1.33 + 0j, 2.7 + 0.05j, 1.48 + 1e-5j, 0.4, 0.55),  # high-index shell
    (0.35, 1.0 + 0j, 1.47 + 0.01j, 1.0 + 0j, 0.25, 0.55),    # fig. 6-like hollow shell
]


@pytest.mark.parametrize("pt", POINTS)
def test_coated_coefficients_vs_mpmath(orc, pt):
    wl, nc, ns, nm, a, b = pt
    o = orc.mie_coated(wl, nc, ns, nm, a, b, with_coeffs=True)
    N = o["n_max"] + 1
    ref = _mp_coated(wl, nc, ns, nm, a, b, N)
    for got, want in ((o["a"], ref[:, 0]), (o["b"], ref[:, 1])):
        scale = np.max(np.abs(want))
        err = np.abs(got - want) / np.maximum(np.abs(want), 1e-6 * scale)
        assert err.max() < 1e-10, err.max()


def test_coated_reduces_to_sphere(orc):
    s = orc.mie_sphere(0.6, 1.5 + 0.01j, 1.33, 0.5, with_coeffs=True)
    same = orc.mie_coated(0.6, 1.5 + 0.01j, 1.5 + 0.01j, 1.33, 0.3, 0.5)
    for k in ("q_ext", "q_sca", "g"):
        assert abs(same[k] - s[k]) < 1e-13 * abs(s[k])
    tiny_core = orc.mie_coated(0.6, 2.5 + 0.1j, 1.5 + 0.01j, 1.33, 1e-6, 0.5)
    assert abs(tiny_core["q_ext"] - s["q_ext"]) < 1e-9 * s["q_ext"]
    core = orc.mie_sphere(0.6, 2.5 + 0.1j, 1.33, 0.5)
    thin_shell = orc.mie_coated(0.6, 2.5 + 0.1j, 1.5 + 0.01j, 1.33, 0.5 - 1e-9, 0.5)
    assert abs(thin_shell["q_ext"] - core["q_ext"]) < 1e-7 * core["q_ext"]


def test_hollow_sphere_conserves_energy(orc):
    for b in (0.3, 0.45, 0.55):
        o = orc.mie_coated(0.5, 1.0 + 0j, 1.45 + 0j, 1.0 + 0j, 0.25, b)
        assert abs(o["q_ext"] - o["q_sca"]) < 1e-11 * o["q_ext"]


def test_coated_effective_medium(orc):
    wl = np.array([0.4, 0.8, 1.6])
    nm = np.array([[1.0 + 0j] * 3, [1.0 + 0j] * 3])
    shell = np.array([[1.45 + 1e-4j] * 3] * 2)
    core = np.array([[1.0 + 0j] * 3] * 2)
    o = orc.mie_properties(wl, nm, [0, 1], shell, [0.35, 0.35], [0.3, 0.3],
                           core_radius=[0.25, 0.0], n_core=core)
    hollow = [orc.mie_coated(w, 1.0, 1.45 + 1e-4j, 1.0, 0.25, 0.35) for w in wl]
    C = 1 + 1.5 * 0.3 - 0.75 * 0.09
    for i, h in enumerate(hollow):
        assert abs(o["mu_s"][0, i] - C * 1.5 * h["q_sca"] * 0.3 / 0.7) < 1e-12 * o["mu_s"][0, i]
    solid = orc.mie_properties(wl, nm[1:], [0], shell[1:], [0.35], [0.3])
    assert np.allclose(o["mu_s"][1], solid["mu_s"][0], rtol=1e-14)
    # a hollow particle scatters less than a solid one of the same outer size
    assert np.all(o["mu_s"][0] < o["mu_s"][1])
