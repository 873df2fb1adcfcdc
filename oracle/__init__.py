"""FOS oracle: plain CPU reference of the hot path (test infrastructure only).

Only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py``'s CPU-baseline leg (and
its reference arm) may import this package.  The product path (the CUDA library and
its Python binding) never imports it and shares no code with it.

Parts:
  * ``fos_oracle.cpp``: Philox4x32-10, the Monte Carlo photon walk (FP64 and an
    FP32 mirror with a fixed operation order), Mie theory for a sphere in an
    absorbing host (Eqs. 1-5, 10-12, 15 of arxiv 2409.00165) and the effective
    medium of Eqs. 13-20, built into ``_build/liboracle.so`` by ``build()``.
  * ``mlp.py``: FP64 NumPy forward and backward pass of the surrogate MLP.

Parity status per function (the pins live in ``tests/test_oracle_*.py``):
  philox4x32_10 ......... pinned (known-answer vectors of the generator's authors)
  neg_log/cos2pi FP32 ... pinned (exhaustive comparison with libm over all inputs)
  hg_cos ................ pinned (sampled mean cosine = g; chi-square vs HG pdf)
  fresnel ............... pinned (normal-incidence closed form, Brewster, TIR,
                          angle-form Fresnel equations)
  mc_run (definition) .. pinned (Beer-Lambert; closed-form Fresnel slab; opaque
                          reflector closed form; two-layer adding; conservation;
                          oblique and conductor closed forms; scattering slabs,
                          the paint layer's optical depths included, vs an
                          independent discrete-ordinates solution of the
                          radiative transfer equation)
  mc_run (FP32 mirror,
   FP64 order) ......... pinned (the same closed forms and solver; agrees with
                          the definition within binomial noise)
  mie_sphere ............ pinned (mpmath 50-digit Bessel evaluation of Eqs. 2-5;
                          Rayleigh limit; optical theorem; phase-function
                          quadrature for g; large-sphere extinction limit)
  mie_properties ........ pinned (hand arithmetic of Eqs. 13-20)
  mie_coated ............ pinned (mpmath 40-digit Bessel J, Y evaluation of Eqs.
                          S1-S9; reduces to the sphere when the core and shell
                          indices are equal, when the core vanishes, and when the
                          shell does)
  size_distribution ..... pinned (volume conserved, symmetry, end/centre weight
                          ratio exp(-4.5), sigma -> 0 limit of the medium)
"""
from __future__ import annotations

import ctypes
import math
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "fos_oracle.cpp")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "liboracle.so")
_lock = threading.Lock()
_lib = None

NCOUNT = 6  # R, A, T, runaway, collisions, interface events
OUT_R, OUT_A, OUT_T, OUT_RUNAWAY = 0, 1, 2, 3


def build(force: bool = False) -> str:
    """Compile the oracle with g++ (no FP contraction, no fast math)."""
    os.makedirs(_BUILD, exist_ok=True)
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    cmd = ["g++", "-O2", "-std=c++17", "-ffp-contract=off", "-fno-fast-math",
           "-fno-strict-aliasing", "-shared", "-fPIC", _SRC, "-o", tmp]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


class OrcBatch(ctypes.Structure):
    _fields_ = [
        ("n_stacks", ctypes.c_int), ("n_wl", ctypes.c_int), ("max_layers", ctypes.c_int),
        ("n_layers", ctypes.c_void_p),
        ("mu_s", ctypes.c_void_p), ("mu_a", ctypes.c_void_p), ("g", ctypes.c_void_p),
        ("n_layer", ctypes.c_void_p), ("thickness", ctypes.c_void_p),
        ("n_above", ctypes.c_void_p), ("n_below", ctypes.c_void_p),
        ("substrate_R", ctypes.c_void_p),
        ("n_photons", ctypes.c_void_p), ("photons_per_item", ctypes.c_longlong),
        ("photon_first", ctypes.c_void_p),
        ("item_list", ctypes.c_void_p), ("n_list", ctypes.c_int),
        ("seed", ctypes.c_ulonglong), ("item_id_base", ctypes.c_uint),
        ("max_events", ctypes.c_longlong),
        ("cos_incidence", ctypes.c_void_p), ("k_below", ctypes.c_void_p),
    ]


def lib():
    global _lib
    with _lock:
        if _lib is None:
            path = build()
            L = ctypes.CDLL(path)
            L.orc_philox4x32_10.argtypes = [ctypes.c_void_p] * 3
            L.orc_uniform.argtypes = [ctypes.c_uint32]
            L.orc_uniform.restype = ctypes.c_double
            L.orc_neg_log_f32.argtypes = [ctypes.c_float]
            L.orc_neg_log_f32.restype = ctypes.c_float
            L.orc_cos2pi_f32.argtypes = [ctypes.c_float]
            L.orc_cos2pi_f32.restype = ctypes.c_float
            L.orc_neg_log_f32_many.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_longlong]
            L.orc_cos2pi_f32_many.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_longlong]
            L.orc_hg_cos_f64.argtypes = [ctypes.c_double, ctypes.c_double]
            L.orc_hg_cos_f64.restype = ctypes.c_double
            L.orc_hg_cos_f32.argtypes = [ctypes.c_float, ctypes.c_float]
            L.orc_hg_cos_f32.restype = ctypes.c_float
            L.orc_fresnel_f64.argtypes = [ctypes.c_double] * 3 + [ctypes.c_void_p]
            L.orc_fresnel_f64.restype = ctypes.c_double
            L.orc_fresnel_conductor_f64.argtypes = [ctypes.c_double] * 4
            L.orc_fresnel_conductor_f64.restype = ctypes.c_double
            L.orc_fresnel_conductor_f32.argtypes = [ctypes.c_float] * 4
            L.orc_fresnel_conductor_f32.restype = ctypes.c_float
            L.orc_solar_weighted.argtypes = ([ctypes.c_int, ctypes.c_int] +
                                             [ctypes.c_void_p] * 4)
            L.orc_mc_run.argtypes = [ctypes.POINTER(OrcBatch), ctypes.c_int, ctypes.c_void_p,
                                     ctypes.c_void_p, ctypes.c_longlong]
            L.orc_mc_run.restype = ctypes.c_int
            L.orc_mie_sphere.argtypes = ([ctypes.c_double] * 6 + [ctypes.c_void_p] * 6
                                         + [ctypes.c_int])
            L.orc_mie_sphere.restype = ctypes.c_int
            L.orc_gamma_term.argtypes = [ctypes.c_double]
            L.orc_gamma_term.restype = ctypes.c_double
            L.orc_log_deriv_psi.argtypes = [ctypes.c_int, ctypes.c_double, ctypes.c_double,
                                            ctypes.c_void_p]
            L.orc_mie_properties.argtypes = ([ctypes.c_int, ctypes.c_void_p, ctypes.c_int,
                                              ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int]
                                             + [ctypes.c_void_p] * 11)
            L.orc_mie_properties.restype = ctypes.c_int
            L.orc_mie_coated.argtypes = [ctypes.c_double] * 9 + [ctypes.c_void_p] * 6 + [ctypes.c_int]
            L.orc_mie_coated.restype = ctypes.c_int
            L.orc_mie_properties_cs.argtypes = ([ctypes.c_int, ctypes.c_void_p, ctypes.c_int,
                                                 ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int]
                                                + [ctypes.c_void_p] * 14)
            L.orc_mie_properties_cs.restype = ctypes.c_int
            _lib = L
    return _lib


def _ptr(a):
    return None if a is None else a.ctypes.data


# ---------------------------------------------------------------------------- RNG
def philox4x32_10(ctr, key):
    c = np.ascontiguousarray(ctr, dtype=np.uint32)
    k = np.ascontiguousarray(key, dtype=np.uint32)
    out = np.zeros(4, dtype=np.uint32)
    lib().orc_philox4x32_10(c.ctypes.data, k.ctypes.data, out.ctypes.data)
    return out


def uniform(x: int) -> float:
    return lib().orc_uniform(int(x) & 0xffffffff)


def neg_log_f32(u: np.ndarray) -> np.ndarray:
    u = np.ascontiguousarray(u, dtype=np.float32)
    out = np.empty_like(u)
    lib().orc_neg_log_f32_many(u.ctypes.data, out.ctypes.data, u.size)
    return out


def cos2pi_f32(u: np.ndarray) -> np.ndarray:
    u = np.ascontiguousarray(u, dtype=np.float32)
    out = np.empty_like(u)
    lib().orc_cos2pi_f32_many(u.ctypes.data, out.ctypes.data, u.size)
    return out


def hg_cos(g: float, u: float, fp32: bool = False) -> float:
    return lib().orc_hg_cos_f32(g, u) if fp32 else lib().orc_hg_cos_f64(g, u)


def fresnel(ni: float, nt: float, ci: float):
    ct = ctypes.c_double(0.0)
    R = lib().orc_fresnel_f64(ni, nt, ci, ctypes.byref(ct))
    return R, ct.value


def fresnel_conductor(ni: float, n2: float, k2: float, ci: float, fp32: bool = False) -> float:
    """Unpolarised reflectance from real index ni into n2 + i k2 at incidence cosine ci."""
    f = lib().orc_fresnel_conductor_f32 if fp32 else lib().orc_fresnel_conductor_f64
    return f(ni, n2, k2, ci)


def solar_weighted(counts, wl, G, n_stacks: int):
    """Eq. 21 totals [n_stacks, 3] (R, A, T) from counts [n_stacks*n_wl, 6]."""
    c = np.ascontiguousarray(counts, dtype=np.int64)
    wl = np.ascontiguousarray(wl, dtype=np.float64)
    G = np.ascontiguousarray(G, dtype=np.float64)
    out = np.zeros((n_stacks, 3))
    lib().orc_solar_weighted(int(n_stacks), int(wl.size), wl.ctypes.data, G.ctypes.data,
                             c.ctypes.data, out.ctypes.data)
    return out


# ---------------------------------------------------------------------------- MC
MODE_F64_ORDER, MODE_F32_MIRROR, MODE_DEFINITION = 0, 1, 2


def mc_run(batch: dict, fp32: bool = True, photon_log: bool = False, mode=None):
    """Run the oracle walk on a batch given as a dict of NumPy arrays.

    mode: MODE_DEFINITION (the walk as the paper states it, FP64, its own sequential
    random stream), MODE_F32_MIRROR (the GPU walk's order and random layout in FP32,
    bit-exact with it) or MODE_F64_ORDER (that order and layout in FP64); None picks
    the mirror if fp32 else the FP64 order.

    Keys mirror the fields of the C-ABI batch (see include/fos.h): n_stacks, n_wl,
    max_layers, n_layers, mu_s, mu_a, g, n_layer, thickness, n_above, n_below,
    substrate_R, n_photons, photons_per_item, photon_first, item_list, seed,
    item_id_base, max_events, cos_incidence, k_below.  Returns int64 counts [n_run, 6] (and the per-photon
    log [n_run, max N] of (collisions << 2 | outcome) when asked).
    """
    keep = []

    def arr(name, dtype):
        v = batch.get(name)
        if v is None:
            return None
        a = np.ascontiguousarray(v, dtype=dtype)
        keep.append(a)
        return a.ctypes.data

    b = OrcBatch()
    b.n_stacks = int(batch["n_stacks"])
    b.n_wl = int(batch["n_wl"])
    b.max_layers = int(batch["max_layers"])
    b.n_layers = arr("n_layers", np.int32)
    for name in ("mu_s", "mu_a", "g", "n_layer", "thickness", "n_above", "n_below",
                 "substrate_R", "cos_incidence", "k_below"):
        setattr(b, name, arr(name, np.float64))
    b.n_photons = arr("n_photons", np.int64)
    b.photons_per_item = int(batch.get("photons_per_item", 0))
    b.photon_first = arr("photon_first", np.int64)
    b.item_list = arr("item_list", np.int32)
    n_items = b.n_stacks * b.n_wl
    b.n_list = int(len(batch["item_list"])) if batch.get("item_list") is not None else 0
    b.seed = int(batch.get("seed", 0))
    b.item_id_base = int(batch.get("item_id_base", 0))
    b.max_events = int(batch.get("max_events", 0))
    n_run = b.n_list if batch.get("item_list") is not None else n_items
    counts = np.zeros((n_run, NCOUNT), dtype=np.int64)
    log = None
    stride = 0
    if photon_log:
        if batch.get("n_photons") is not None:
            stride = int(np.max(batch["n_photons"])) if n_items else 0
        else:
            stride = b.photons_per_item
        log = np.full((n_run, max(stride, 1)), -1, dtype=np.int32)
    if mode is None:
        mode = MODE_F32_MIRROR if fp32 else MODE_F64_ORDER
    rc = lib().orc_mc_run(ctypes.byref(b), int(mode), counts.ctypes.data,
                          _ptr(log), stride)
    if rc != 0:
        raise ValueError(f"oracle mc_run rejected the batch (code {rc})")
    return (counts, log) if photon_log else counts


def mc_run_threads(batch: dict, mode: int = MODE_DEFINITION, threads: int = 0):
    """mc_run split over host threads by photon range (the library call releases the
    GIL); counts depend only on photon ids, so the shard sums equal one run exactly."""
    from concurrent.futures import ThreadPoolExecutor
    threads = threads or (os.cpu_count() or 1)
    n_items = int(batch["n_stacks"]) * int(batch["n_wl"])
    if batch.get("n_photons") is not None:
        N = np.asarray(batch["n_photons"], np.int64).reshape(-1)
    else:
        N = np.full(n_items, int(batch.get("photons_per_item", 0)), np.int64)
    first0 = (np.zeros(n_items, np.int64) if batch.get("photon_first") is None
              else np.asarray(batch["photon_first"], np.int64).reshape(-1))
    shards = []
    for t in range(threads):
        lo = N * t // threads
        hi = N * (t + 1) // threads
        b = dict(batch)
        b["n_photons"] = hi - lo
        b["photon_first"] = first0 + lo
        b.pop("photons_per_item", None)
        shards.append(b)
    with ThreadPoolExecutor(max_workers=threads) as ex:
        parts = list(ex.map(lambda b: mc_run(b, mode=mode), shards))
    return sum(parts)


# ---------------------------------------------------------------------------- Mie
def mie_sphere(wl, n_p, n_m, r, with_coeffs: bool = False):
    """Q_ext, Q_sca, g (and a_n, b_n for n = 1..n_max+1) of one sphere."""
    qe, qs, gg = ctypes.c_double(), ctypes.c_double(), ctypes.c_double()
    nmax = ctypes.c_int()
    cap = 2048
    an = np.zeros(2 * cap) if with_coeffs else None
    bn = np.zeros(2 * cap) if with_coeffs else None
    lib().orc_mie_sphere(float(wl), float(np.real(n_p)), float(np.imag(n_p)), float(np.real(n_m)),
                         float(np.imag(n_m)), float(r), ctypes.byref(qe), ctypes.byref(qs),
                         ctypes.byref(gg), ctypes.byref(nmax), _ptr(an), _ptr(bn), cap)
    out = dict(q_ext=qe.value, q_sca=qs.value, g=gg.value, n_max=nmax.value)
    if with_coeffs:
        k = nmax.value + 1
        out["a"] = an[: 2 * k].view(np.complex128).copy()
        out["b"] = bn[: 2 * k].view(np.complex128).copy()
    return out


def size_distribution(diameter, sigma, vol_frac, n=101):
    """Section "Scattering properties", last paragraph: a diameter with standard
    deviation sigma becomes n diameters over D +- 3 sigma; the volume fraction is shared
    by Gaussian weights (normalised); non-positive diameters are dropped.  Plain Python."""
    if sigma == 0 or n == 1:
        return np.array([diameter / 2.0]), np.array([float(vol_frac)])
    ds, ws = [], []
    for i in range(n):
        d = diameter - 3.0 * sigma + 6.0 * sigma * i / (n - 1)
        if d <= 0:
            continue
        ds.append(d / 2.0)
        ws.append(math.exp(-0.5 * ((d - diameter) / sigma) ** 2))
    tot = sum(ws)
    return np.array(ds), np.array([vol_frac * w / tot for w in ws])


def mie_coated(wl, n_core, n_shell, n_m, a, b, with_coeffs: bool = False):
    """Q_ext, Q_sca, g (and a_n, b_n) of a core-shell sphere (Eqs. S1-S9)."""
    qe, qs, gg = ctypes.c_double(), ctypes.c_double(), ctypes.c_double()
    nmax = ctypes.c_int()
    cap = 2048
    an = np.zeros(2 * cap) if with_coeffs else None
    bn = np.zeros(2 * cap) if with_coeffs else None
    lib().orc_mie_coated(float(wl), float(np.real(n_core)), float(np.imag(n_core)),
                         float(np.real(n_shell)), float(np.imag(n_shell)), float(np.real(n_m)),
                         float(np.imag(n_m)), float(a), float(b), ctypes.byref(qe), ctypes.byref(qs),
                         ctypes.byref(gg), ctypes.byref(nmax), _ptr(an), _ptr(bn), cap)
    out = dict(q_ext=qe.value, q_sca=qs.value, g=gg.value, n_max=nmax.value)
    if with_coeffs:
        k = nmax.value + 1
        out["a"] = an[: 2 * k].view(np.complex128).copy()
        out["b"] = bn[: 2 * k].view(np.complex128).copy()
    return out


def gamma_term(alpha: float) -> float:
    return lib().orc_gamma_term(float(alpha))


def log_deriv_psi(n: int, z: complex) -> complex:
    out = np.zeros(2)
    lib().orc_log_deriv_psi(int(n), float(np.real(z)), float(np.imag(z)), out.ctypes.data)
    return complex(out[0], out[1])


def mie_properties(wl, nm, species_group, n_p, radius, vol_frac, n_groups=None,
                   core_radius=None, n_core=None):
    """Effective-medium mu_s, mu_a, g per (group, wavelength) and per-species Q's.

    wl [n_wl]; nm complex [n_groups, n_wl]; n_p complex [n_species, n_wl] (the shell of
    a core-shell species); species_group, radius (outer), vol_frac [n_species]; optional
    core_radius [n_species] (> 0: core-shell) and n_core complex [n_species, n_wl].
    """
    wl = np.ascontiguousarray(wl, dtype=np.float64)
    nm = np.asarray(nm, dtype=np.complex128)
    n_p = np.asarray(n_p, dtype=np.complex128)
    n_wl = wl.size
    n_groups = nm.shape[0] if n_groups is None else n_groups
    n_species = len(radius)
    nm_re = np.ascontiguousarray(nm.real.reshape(-1))
    nm_im = np.ascontiguousarray(nm.imag.reshape(-1))
    np_re = np.ascontiguousarray(n_p.real.reshape(-1))
    np_im = np.ascontiguousarray(n_p.imag.reshape(-1))
    sg = np.ascontiguousarray(species_group, dtype=np.int32)
    rad = np.ascontiguousarray(radius, dtype=np.float64)
    vf = np.ascontiguousarray(vol_frac, dtype=np.float64)
    mu_s = np.zeros(n_groups * n_wl)
    mu_a = np.zeros(n_groups * n_wl)
    g = np.zeros(n_groups * n_wl)
    qe = np.zeros(n_species * n_wl)
    qs = np.zeros(n_species * n_wl)
    gs = np.zeros(n_species * n_wl)
    if core_radius is None:
        lib().orc_mie_properties(n_wl, wl.ctypes.data, n_groups, nm_re.ctypes.data,
                                 nm_im.ctypes.data, n_species, sg.ctypes.data, np_re.ctypes.data,
                                 np_im.ctypes.data, rad.ctypes.data, vf.ctypes.data,
                                 mu_s.ctypes.data, mu_a.ctypes.data, g.ctypes.data,
                                 qe.ctypes.data, qs.ctypes.data, gs.ctypes.data)
    else:
        nc = np.asarray(n_core, dtype=np.complex128)
        nc_re = np.ascontiguousarray(nc.real.reshape(-1))
        nc_im = np.ascontiguousarray(nc.imag.reshape(-1))
        cr = np.ascontiguousarray(core_radius, dtype=np.float64)
        lib().orc_mie_properties_cs(n_wl, wl.ctypes.data, n_groups, nm_re.ctypes.data,
                                    nm_im.ctypes.data, n_species, sg.ctypes.data,
                                    np_re.ctypes.data, np_im.ctypes.data, nc_re.ctypes.data,
                                    nc_im.ctypes.data, rad.ctypes.data, cr.ctypes.data,
                                    vf.ctypes.data, mu_s.ctypes.data, mu_a.ctypes.data,
                                    g.ctypes.data, qe.ctypes.data, qs.ctypes.data,
                                    gs.ctypes.data)
    shp = (n_groups, n_wl)
    sshp = (n_species, n_wl)
    return dict(mu_s=mu_s.reshape(shp), mu_a=mu_a.reshape(shp), g=g.reshape(shp),
                q_ext=qe.reshape(sshp), q_sca=qs.reshape(sshp), g_sp=gs.reshape(sshp))
