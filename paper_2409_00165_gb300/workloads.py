"""Seeded synthetic workloads for FOS (arxiv 2409.00165): inputs only.

This module builds the inputs of the five standard workloads as NumPy arrays in
the layouts of the C-ABI (include/fos.h).  It holds none of the method's
arithmetic (no Mie theory, no effective medium, no photon transport): only
wavelength grids, synthetic material indices and seeded design draws.  Both the
CUDA path and the CPU oracle take their inputs from here.

The paper's own material files (BaSO4, TiO2, acrylic, ...) are not available, so
the materials are closed-form stand-ins:
  * particle: Cauchy n = 2.5 + 0.05/lambda^2 (lambda in um), k = 0.5 below
    0.4 um and 1e-4 from 0.4 um on (a TiO2-like absorption edge);
  * matrix: n = 1.48, k = 1e-5 * lambda (an acrylic-like weakly absorbing binder).
Layer index arrays are laid out per group g = stack * max_layers + layer.
"""
from __future__ import annotations

import numpy as np

# Photon budgets and sizes of the standard workloads.
PAINT_N_WL = 400          # full-spectrum paint layer
STACK_N_DESIGNS = 64      # uneven multilayer batch
STACK_N_WL = 200
SWEEP_N_WL = 300          # surrogate design sweep


def wavelengths(n: int, lo: float = 0.3, hi: float = 2.5) -> np.ndarray:
    """Uniform vacuum-wavelength grid in um, both ends included."""
    return np.linspace(lo, hi, n)


def particle_index(wl: np.ndarray) -> np.ndarray:
    wl = np.asarray(wl, dtype=np.float64)
    n = 2.5 + 0.05 / (wl * wl)
    k = np.where(wl < 0.4, 0.5, 1e-4)
    return n + 1j * k


def matrix_index(wl: np.ndarray) -> np.ndarray:
    wl = np.asarray(wl, dtype=np.float64)
    return 1.48 + 1j * (1e-5 * wl)


# --------------------------------------------------------------------------------
# Single slab with given optical properties (no Mie): 0.5 mm, mu_s = 10/mm,
# mu_a = 0.1/mm, g = 0.7, n = 1.5 in air, 1e5 photons, seed 1.
# --------------------------------------------------------------------------------
def single_slab(n_photons: int = 100000, seed: int = 1, mu_s: float = 10.0,
                mu_a: float = 0.1, g: float = 0.7, n: float = 1.5, d: float = 0.5,
                n_above: float = 1.0, n_below: float = 1.0) -> dict:
    return dict(n_stacks=1, n_wl=1, max_layers=1,
                n_layers=np.array([1], np.int32),
                mu_s=np.array([mu_s]), mu_a=np.array([mu_a]), g=np.array([g]),
                n_layer=np.array([n]), thickness=np.array([d]),
                n_above=np.array([n_above]), n_below=np.array([n_below]),
                substrate_R=None, n_photons=None, photons_per_item=int(n_photons),
                photon_first=None, item_list=None, seed=int(seed), item_id_base=0,
                max_events=0)


# --------------------------------------------------------------------------------
# Particle media described for Mie + effective medium, then photon transport.
# --------------------------------------------------------------------------------
def _media(wl, radius, vol_frac, thickness, n_layers, max_layers):
    """Species/group tables for stacks whose layers hold one particle species each.

    radius, vol_frac, thickness: [n_stacks, max_layers]; n_layers: [n_stacks].
    """
    n_stacks = len(n_layers)
    n_wl = len(wl)
    n_groups = n_stacks * max_layers
    nm = np.broadcast_to(matrix_index(wl), (n_groups, n_wl)).copy()
    sg, rad, vf = [], [], []
    for s in range(n_stacks):
        for j in range(int(n_layers[s])):
            sg.append(s * max_layers + j)
            rad.append(radius[s, j])
            vf.append(vol_frac[s, j])
    n_species = len(sg)
    n_p = np.broadcast_to(particle_index(wl), (n_species, n_wl)).copy()
    return dict(wl=np.asarray(wl, np.float64), n_groups=n_groups, nm=nm,
                species_group=np.array(sg, np.int32), n_p=n_p,
                radius=np.array(rad, np.float64), vol_frac=np.array(vf, np.float64),
                thickness=np.asarray(thickness, np.float64).reshape(-1),
                n_layers=np.asarray(n_layers, np.int32), n_stacks=n_stacks,
                max_layers=max_layers, n_wl=n_wl)


def paint_layer(n_wl: int = PAINT_N_WL, photons: int = 1000000, seed: int = 1,
                radius: float = 0.2, vol_frac: float = 0.10,
                thickness: float = 300.0) -> dict:
    """Full-spectrum paint layer: one 300 um layer, r = 0.2 um, f = 0.10, air both sides."""
    wl = wavelengths(n_wl)
    m = _media(wl, np.array([[radius]]), np.array([[vol_frac]]), np.array([[thickness]]),
               np.array([1]), 1)
    m.update(photons_per_item=int(photons), n_photons=None, substrate_R=None,
             seed=int(seed))
    return m


def layer_stacks(n_designs: int = STACK_N_DESIGNS, n_wl: int = STACK_N_WL, seed: int = 3,
                 substrate_R: float = 0.05, photons_lo: float = 1e4,
                 photons_hi: float = 1e6) -> dict:
    """Uneven batch of 1-3 layer stacks on an opaque reflector.

    Per layer r ~ U(0.05, 1) um, f ~ U(0.01, 0.3), d ~ U(10, 500) um; photon budgets
    round(10^U(log10 lo, log10 hi)) per (design, wavelength); numpy default_rng(seed).
    """
    rng = np.random.default_rng(seed)
    max_layers = 3
    n_layers = rng.integers(1, 4, size=n_designs)
    radius = rng.uniform(0.05, 1.0, size=(n_designs, max_layers))
    vol_frac = rng.uniform(0.01, 0.3, size=(n_designs, max_layers))
    thickness = rng.uniform(10.0, 500.0, size=(n_designs, max_layers))
    wl = wavelengths(n_wl)
    m = _media(wl, radius, vol_frac, thickness, n_layers, max_layers)
    budgets = np.round(10.0 ** rng.uniform(np.log10(photons_lo), np.log10(photons_hi),
                                           size=n_designs * n_wl)).astype(np.int64)
    m.update(n_photons=budgets, photons_per_item=0,
             substrate_R=np.full(n_designs * n_wl, float(substrate_R)), seed=int(seed))
    return m


def single_layer_designs(n_designs: int, seed: int, n_wl: int | None = SWEEP_N_WL,
                         random_wl: bool = False, log_share: float = 0.0) -> dict:
    """Single-layer designs in the ranges of the multilayer batch (r, f, d), uniform.

    With random_wl, each design gets one wavelength drawn from U(0.3, 2.5) um; otherwise
    every design uses the n_wl-point grid.  A fraction log_share of the designs draws f
    and d log-uniformly over the same ranges instead, which puts more of them near the
    thin, dilute end (a training-set choice: the sweep itself is uniform).
    """
    rng = np.random.default_rng(seed)
    radius = rng.uniform(0.05, 1.0, size=n_designs)
    vol_frac = rng.uniform(0.01, 0.3, size=n_designs)
    thickness = rng.uniform(10.0, 500.0, size=n_designs)
    if log_share > 0.0:
        pick = rng.uniform(size=n_designs) < log_share
        lf = np.exp(rng.uniform(np.log(0.01), np.log(0.3), size=n_designs))
        ld = np.exp(rng.uniform(np.log(10.0), np.log(500.0), size=n_designs))
        vol_frac = np.where(pick, lf, vol_frac)
        thickness = np.where(pick, ld, thickness)
    if random_wl:
        wl = rng.uniform(0.3, 2.5, size=n_designs)
    elif n_wl:
        wl = wavelengths(n_wl)
    else:
        wl = None
    return dict(radius=radius, vol_frac=vol_frac, thickness=thickness, wl=wl,
                random_wl=bool(random_wl))


def media_arrays(m: dict) -> dict:
    """Matrix and particle indices split into real and imaginary parts."""
    return dict(nm_re=np.ascontiguousarray(m["nm"].real.reshape(-1)),
                nm_im=np.ascontiguousarray(m["nm"].imag.reshape(-1)),
                np_re=np.ascontiguousarray(m["n_p"].real.reshape(-1)),
                np_im=np.ascontiguousarray(m["n_p"].imag.reshape(-1)))


# --------------------------------------------------------------------------------
# Size distributions: silicon-like particles in water (the paper's Si-water example
# with synthetic materials): D = 0.5 um at volume fraction 0.1 %, standard deviations
# 0, 0.05, 0.15 um, a 500 um layer, 400 wavelengths.
# --------------------------------------------------------------------------------
def silicon_like_index(wl):
    """n = 3.45 + 0.2/lambda^2, k = 0.5 exp(-(lambda - 0.3)/0.1) (an absorption edge)."""
    wl = np.asarray(wl, dtype=np.float64)
    return (3.45 + 0.2 / (wl * wl)) + 1j * (0.5 * np.exp(-(wl - 0.3) / 0.1))


def water_like_index(wl):
    """n = 1.33, k = 1e-7 + 1e-5 lambda^4 (absorption rising into the infrared)."""
    wl = np.asarray(wl, dtype=np.float64)
    return 1.33 + 1j * (1e-7 + 1e-5 * wl ** 4)


def size_distribution_media(distributions, diameter=0.5, vol_frac=0.001, thickness=500.0,
                            n_wl=PAINT_N_WL, n_sizes=101):
    """One single-layer stack per standard deviation in `distributions`.  The expansion
    of each distribution into sizes is passed in as `distributions`:
    a list of (radius array, vol_frac array) pairs (see fos_size_distribution)."""
    wl = wavelengths(n_wl)
    sg, rad, vf = [], [], []
    for s, (r, f) in enumerate(distributions):
        sg += [s] * len(r)
        rad += list(r)
        vf += list(f)
    n_groups = len(distributions)
    nm = np.broadcast_to(water_like_index(wl), (n_groups, n_wl)).copy()
    n_p = np.broadcast_to(silicon_like_index(wl), (len(rad), n_wl)).copy()
    return dict(wl=wl, n_groups=n_groups, nm=nm, species_group=np.array(sg, np.int32),
                n_p=n_p, radius=np.array(rad), vol_frac=np.array(vf),
                thickness=np.full(n_groups, float(thickness)),
                n_layers=np.ones(n_groups, np.int32), n_stacks=n_groups, max_layers=1,
                n_wl=n_wl)


# --------------------------------------------------------------------------------
# Core-shell particles: the paper's hollow-SiO2 example with a synthetic silica.
# Hollow spheres (air core of diameter 0.5 um) of outer diameter 0.7, 0.9, 1.1 um, and
# solid spheres of the same outer diameters, at volume fraction 0.6 in a 50 um layer in
# air; 400 wavelengths over 0.3-2.5 um.
# --------------------------------------------------------------------------------
def silica_like_index(wl):
    """n = sqrt(1 + 1.1 lambda^2 / (lambda^2 - 0.01)), k = 1e-6 + 1e-4 (lambda / 2.5)^4
    (a one-term Sellmeier form near 1.45 with weak absorption rising to the infrared)."""
    wl = np.asarray(wl, dtype=np.float64)
    l2 = wl * wl
    return np.sqrt(1.0 + 1.1 * l2 / (l2 - 0.01)) + 1j * (1e-6 + 1e-4 * (wl / 2.5) ** 4)


def hollow_silica_media(outer_diameters=(0.7, 0.9, 1.1), core_diameter=0.5, vol_frac=0.6,
                        thickness=50.0, n_wl=PAINT_N_WL, solid=True):
    """One single-layer stack per outer diameter with hollow silica spheres, then (solid)
    one per outer diameter with solid silica spheres.  Adds core_radius (0 for solid)
    and n_core [n_species, n_wl] (air) to the media dict."""
    wl = wavelengths(n_wl)
    outer = list(outer_diameters)
    radius = [0.5 * d for d in outer] + ([0.5 * d for d in outer] if solid else [])
    core = [0.5 * core_diameter] * len(outer) + ([0.0] * len(outer) if solid else [])
    n_groups = len(radius)
    nm = np.ones((n_groups, n_wl), np.complex128)
    n_p = np.broadcast_to(silica_like_index(wl), (n_groups, n_wl)).copy()
    return dict(wl=wl, n_groups=n_groups, nm=nm, species_group=np.arange(n_groups, dtype=np.int32),
                n_p=n_p, n_core=np.ones((n_groups, n_wl), np.complex128),
                radius=np.array(radius), core_radius=np.array(core),
                vol_frac=np.full(n_groups, float(vol_frac)),
                thickness=np.full(n_groups, float(thickness)),
                n_layers=np.ones(n_groups, np.int32), n_stacks=n_groups, max_layers=1,
                n_wl=n_wl)


# --------------------------------------------------------------------------------
# Boundary and incidence variants, and the solar weighting of Eq. 21.  The AM1.5
# spectrum file is not available: a 5778 K blackbody shape stands in for G.
# --------------------------------------------------------------------------------
def solar_like_irradiance(wl):
    """Planck spectral shape at 5778 K, lambda in um (arbitrary scale, peak ~1)."""
    wl = np.asarray(wl, dtype=np.float64)
    c2 = 14387.77   # um K
    b = wl ** -5 / np.expm1(c2 / (wl * 5778.0))
    return b / (0.5 ** -5 / np.expm1(c2 / (0.5 * 5778.0)))


def aluminium_like_index(wl):
    """Drude metal n + ik = sqrt(1 - (lambda/0.083)^2 / (1 + i lambda/12.4)), lambda in
    um (plasma wavelength 0.083 um, damping wavelength 12.4 um)."""
    wl = np.asarray(wl, dtype=np.float64)
    eps = 1.0 - (wl / 0.083) ** 2 / (1.0 + 1j * wl / 12.4)
    n = np.sqrt(eps.astype(np.complex128))
    return np.where(n.imag < 0, -n, n)


def oblique_conductor_media(cos_incidence=(1.0, 0.8660254037844387, 0.5), n_wl=PAINT_N_WL,
                            thickness=50.0, radius=0.2, vol_frac=0.10):
    """The paint-layer medium, 50 um thick, on an aluminium-like conductor, lit at 0, 30
    and 60 degrees: one single-layer stack per incidence angle.  Adds per-item
    cos_incidence, n_below and k_below arrays [n_stacks * n_wl]."""
    wl = wavelengths(n_wl)
    k = len(cos_incidence)
    m = _media(wl, np.full((k, 1), radius), np.full((k, 1), vol_frac),
               np.full((k, 1), thickness), np.ones(k, np.int32), 1)
    al = aluminium_like_index(wl)
    m.update(cos_incidence=np.repeat(np.asarray(cos_incidence, np.float64), n_wl),
             n_below=np.tile(al.real, k), k_below=np.tile(al.imag, k))
    return m


# --------------------------------------------------------------------------------
# Slabs given by optical properties, for the network with the paper's inputs (Table 1):
# matrix index 1-7, mu_a 0-1e6 /cm, mu_s 0-2e5 /cm, g 0-1, thickness 5-500 um, air on
# both sides.  Units here: 1/um and um (1e6 /cm = 100 /um, 2e5 /cm = 20 /um).  The
# scattering optical depth is capped at 100: beyond it a walk takes ~tau^2 steps per
# photon, which no training budget affords.
# --------------------------------------------------------------------------------
TABLE1 = dict(n=(1.0, 7.0), mu_s=(0.0, 20.0), mu_a=(0.0, 100.0), g=(0.0, 0.99),
              d=(5.0, 500.0), tau_s_max=100.0)


def table1_slabs(n_rows: int, seed: int, tau_s_max: float = TABLE1["tau_s_max"],
                 zero_frac: float = 0.05, g_log_share: float = 0.0,
                 n_log_share: float = 0.0) -> dict:
    """n ~ U(1, 7), g ~ U(0, 0.99), d log-uniform on [5, 500] um, mu_s log-uniform on
    [1e-4, min(20, tau_s_max / d)] /um, mu_a log-uniform on [1e-4, 100] /um; a fraction
    zero_frac of rows has mu_s = 0 and another mu_a = 0 (the lower ends of Table 1).  A
    fraction g_log_share of the rows draws 1 - g log-uniformly on [0.01, 1] instead,
    which puts more of them near g = 1, and a fraction n_log_share draws n - 1
    log-uniformly on [1e-3, 6], which puts more of them near an index-matched slab
    (training-set choices)."""
    rng = np.random.default_rng(seed)
    lo, hi = np.log(1e-4), np.log(20.0)
    d = np.exp(rng.uniform(np.log(5.0), np.log(500.0), n_rows))
    top = np.log(np.minimum(20.0, tau_s_max / d))
    mu_s = np.exp(lo + rng.uniform(size=n_rows) * (top - lo))
    mu_a = np.exp(rng.uniform(np.log(1e-4), np.log(100.0), n_rows))
    mu_s[rng.uniform(size=n_rows) < zero_frac] = 0.0
    mu_a[rng.uniform(size=n_rows) < zero_frac] = 0.0
    n = rng.uniform(1.0, 7.0, n_rows)
    g = rng.uniform(0.0, 0.99, n_rows)
    if g_log_share > 0.0:
        pick = rng.uniform(size=n_rows) < g_log_share
        g = np.where(pick, 1.0 - np.exp(rng.uniform(np.log(0.01), 0.0, n_rows)), g)
    if n_log_share > 0.0:
        pick = rng.uniform(size=n_rows) < n_log_share
        n = np.where(pick, 1.0 + np.exp(rng.uniform(np.log(1e-3), np.log(6.0), n_rows)), n)
    return dict(n=n, mu_s=mu_s, mu_a=mu_a, g=g, d=d)
