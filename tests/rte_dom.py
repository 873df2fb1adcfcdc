"""Deterministic solution of the radiative transfer equation in a plane slab.

An independent pin for the Monte Carlo walk: the azimuthally averaged RTE

    mu dI/dtau = -I + (omega/2) int_{-1}^{1} p0(mu, mu') I(mu') dmu' + Q(tau, mu)

for a homogeneous slab of optical thickness tau_d, single-scattering albedo omega and
a Henyey-Greenstein phase function, lit by a collimated beam (normal or oblique
incidence; the azimuthally averaged equation carries the fluxes either way).
The discrete-ordinates method (Chandrasekhar; Stamnes et al. 1988) replaces the
integral by Gauss-Legendre quadrature, solves the homogeneous system by eigen-
decomposition (exponentials scaled so that none overflows) and the collimated
source by its particular solution.  Specular Fresnel boundaries are exact in this
frame because reflection keeps the direction cosine; total internal reflection is
resolved by splitting the quadrature at the critical cosine.

The unscattered beam and its specular bounces are summed in closed form.  Fresnel
reflectance here uses the angle form R = (sin^2(ti-tt)/sin^2(ti+tt) +
tan^2(ti-tt)/tan^2(ti+tt))/2, a different expression from the one in the walk.
Returns (R, A, T) as fractions of the incident flux.
"""
from __future__ import annotations

import numpy as np


def fresnel_angle_form(n_i: float, n_t: float, mu_i: np.ndarray) -> np.ndarray:
    mu_i = np.asarray(mu_i, dtype=np.float64)
    out = np.ones_like(mu_i)
    if n_i == n_t:
        return np.zeros_like(mu_i)
    ti = np.arccos(np.clip(mu_i, -1.0, 1.0))
    st = n_i / n_t * np.sin(ti)
    ok = st < 1.0
    tt = np.arcsin(np.where(ok, st, 0.0))
    normal = ok & (ti < 1e-7)
    rn = ((n_i - n_t) / (n_i + n_t)) ** 2
    with np.errstate(divide="ignore", invalid="ignore"):
        rs = np.sin(ti - tt) ** 2 / np.sin(ti + tt) ** 2
        rp = np.tan(ti - tt) ** 2 / np.tan(ti + tt) ** 2
    val = 0.5 * (rs + rp)
    out = np.where(ok, val, 1.0)
    out = np.where(normal, rn, out)
    return out


def fresnel_complex_angle_form(n_i: float, n_t: complex, mu_i: np.ndarray) -> np.ndarray:
    """Reflectance into an absorbing medium n_t = n + ik: Snell's law with complex
    angles and the sine/tangent forms (normal incidence: |(n_i - n_t)/(n_i + n_t)|^2)."""
    mu_i = np.asarray(mu_i, dtype=np.float64)
    ti = np.arccos(np.clip(mu_i, -1.0, 1.0))
    tt = np.arcsin(n_i * np.sin(ti) / n_t + 0j)
    with np.errstate(divide="ignore", invalid="ignore"):
        rs = np.abs(np.sin(ti - tt) / np.sin(ti + tt)) ** 2
        rp = np.abs(np.tan(ti - tt) / np.tan(ti + tt)) ** 2
    rn = abs((n_i - n_t) / (n_i + n_t)) ** 2
    return np.where(ti < 1e-7, rn, 0.5 * (rs + rp))


def _hg(g: float, c: np.ndarray) -> np.ndarray:
    return (1.0 - g * g) / (1.0 + g * g - 2.0 * g * c) ** 1.5


def _nodes(n_in: float, n_out_top: float, n_out_bot: float, n_half: int):
    """Gauss-Legendre nodes on (0, 1], split at the critical cosines."""
    cuts = [0.0, 1.0]
    for n_out in (n_out_top, n_out_bot):
        if n_out < n_in:
            cuts.append(float(np.sqrt(1.0 - (n_out / n_in) ** 2)))
    cuts = sorted(set(cuts))
    spans = np.diff(cuts)
    per = [max(4, int(round(n_half * s))) for s in spans]
    mus, ws = [], []
    for (a, b), m in zip(zip(cuts[:-1], cuts[1:]), per):
        x, w = np.polynomial.legendre.leggauss(m)
        mus.append(0.5 * (b - a) * x + 0.5 * (b + a))
        ws.append(0.5 * (b - a) * w)
    return np.concatenate(mus), np.concatenate(ws)


def slab_rat(mu_s: float, mu_a: float, g: float, d: float, n_in: float,
             n_above: float = 1.0, n_below: float = 1.0, n_half: int = 48,
             n_phi: int = 720, mu0: float = 1.0, k_below: float = 0.0):
    """(R, A, T) for a beam at incidence cosine mu0 from above (refracted to mu_in in
    the slab); k_below > 0 makes the medium below absorbing (n_below + i k_below),
    whose entering flux counts as T."""
    mu_t = mu_s + mu_a
    tau_d = mu_t * d
    omega = mu_s / mu_t if mu_t > 0 else 0.0
    conductor = k_below > 0.0
    mu, w = _nodes(n_in, n_above, n_in if conductor else n_below, n_half)
    if conductor:
        rbot = lambda m: fresnel_complex_angle_form(n_in, complex(n_below, k_below), m)
    else:
        rbot = lambda m: fresnel_angle_form(n_in, n_below, m)
    st_in = n_above / n_in * np.sqrt(max(0.0, 1.0 - mu0 * mu0))
    if st_in >= 1.0:
        return 1.0, 0.0, 0.0
    mu_in = float(np.sqrt(1.0 - st_in * st_in))
    N = mu.size
    # Azimuthally averaged phase function on the grid (periodic trapezoid in phi).
    phi = (np.arange(n_phi) + 0.5) * (2.0 * np.pi / n_phi)
    cphi = np.cos(phi)
    sgn_mu = np.concatenate([mu, -mu])            # + down, - up
    wt = np.concatenate([w, w])
    s = np.sqrt(np.maximum(0.0, 1.0 - sgn_mu ** 2))
    cos_t = (sgn_mu[:, None, None] * sgn_mu[None, :, None]
             + s[:, None, None] * s[None, :, None] * cphi[None, None, :])
    p0 = _hg(g, cos_t).mean(axis=2)
    # Renormalise each row so that the discrete phase function conserves energy.
    p0 *= 2.0 / (p0 @ wt)[:, None]
    # dI/dtau = M I + source
    M = (-np.eye(2 * N) + 0.5 * omega * p0 * wt[None, :]) / sgn_mu[:, None]
    # Unscattered beam with all its specular bounces, at mu_in inside the slab; D, U are
    # its downward and upward fluxes through horizontal planes.
    r_top_in = fresnel_angle_form(n_above, n_in, np.array([mu0]))[0]
    r_t = fresnel_angle_form(n_in, n_above, np.array([mu_in]))[0]
    r_b = rbot(np.array([mu_in]))[0]
    F0 = 1.0 - r_top_in
    e_d = np.exp(-tau_d / mu_in)
    D0 = F0 / (1.0 - r_t * r_b * e_d * e_d)       # D(tau) = D0 e^{-tau/mu_in}
    U0 = r_b * D0 * e_d                           # U(tau) = U0 e^{-(tau_d - tau)/mu_in}
    # Beam source (omega/4pi)(flux/mu_in) p0(mu, +-mu_in), p0 the azimuthal mean of HG
    s_in = np.sqrt(max(0.0, 1.0 - mu_in * mu_in))
    p_dn = _hg(g, sgn_mu[:, None] * mu_in + s[:, None] * s_in * cphi[None, :]).mean(axis=1)
    p_up = _hg(g, -sgn_mu[:, None] * mu_in + s[:, None] * s_in * cphi[None, :]).mean(axis=1)
    s1 = omega / (4 * np.pi) * D0 / mu_in * p_dn / sgn_mu
    s2 = omega / (4 * np.pi) * U0 / mu_in * p_up / sgn_mu
    I2 = np.eye(2 * N)
    c1 = np.linalg.solve(-(I2 / mu_in + M), s1)   # particular part of e^{-tau/mu_in}
    c2 = np.linalg.solve(I2 / mu_in - M, s2)      # particular part of e^{(tau - tau_d)/mu_in}
    lam, V = np.linalg.eig(M)
    neg = lam.real < 0

    def homog(tau):
        # columns: v_k e^{lam_k tau} (lam<0) and v_k e^{lam_k (tau - tau_d)} (lam>0)
        ex = np.exp(np.where(neg, lam * tau, lam * (tau - tau_d)))
        return V * ex[None, :]

    Rf_top = fresnel_angle_form(n_in, n_above, mu)
    Rf_bot = rbot(mu)
    H0, Hd = homog(0.0), homog(tau_d)
    P0 = c1 + c2 * e_d
    Pd = c1 * e_d + c2
    # tau = 0: I(+mu) - Rf_top I(-mu) = 0; tau = tau_d: I(-mu) - Rf_bot I(+mu) = 0
    A = np.zeros((2 * N, 2 * N), dtype=complex)
    b = np.zeros(2 * N, dtype=complex)
    A[:N] = H0[:N] - Rf_top[:, None] * H0[N:]
    b[:N] = -(P0[:N] - Rf_top * P0[N:])
    A[N:] = Hd[N:] - Rf_bot[:, None] * Hd[:N]
    b[N:] = -(Pd[N:] - Rf_bot * Pd[:N])
    coef = np.linalg.solve(A, b)
    I0 = (H0 @ coef).real + P0
    Id = (Hd @ coef).real + Pd
    up0 = I0[N:]
    dnd = Id[:N]
    R_diff = 2 * np.pi * np.sum(w * mu * (1.0 - Rf_top) * up0)
    T_diff = 2 * np.pi * np.sum(w * mu * (1.0 - Rf_bot) * dnd)
    R = r_top_in + U0 * e_d * (1.0 - r_t) + R_diff
    T = D0 * e_d * (1.0 - r_b) + T_diff
    return float(R), float(1.0 - R - T), float(T)
