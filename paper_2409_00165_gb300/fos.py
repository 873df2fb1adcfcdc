"""Thin Python binding of libfos (include/fos.h): argument marshalling only.

Every function has the name of the C entry point it calls and takes CUDA torch tensors
(PyTorch supplies device memory and streams).  Nothing here computes: every step runs
in the library's kernels.  If libfos.so cannot be loaded the calls raise, there is no
fallback.
"""
from __future__ import annotations

import ctypes
import os
import threading

import torch

from . import build as _build

FOS_OK = 0
FOS_ERR_INVALID_ARG = 1
FOS_ERR_CUDA = 2
FOS_ERR_NOMEM = 3
FOS_ERR_STEP_LIMIT = 4
FOS_ERR_TIMEOUT = 5
FOS_ERR_OUT_OF_RANGE = 6
FOS_ERR_INJECTED = 7
FOS_ERR_UNSUPPORTED = 8

FOS_ASYNC = 0x1
FOS_NO_GRAPH = 0x2
FOS_AUTOTUNE = 0x4
FOS_FAST_WALK = 0x8
FOS_RECORD_TIMES = 0x10
FOS_TEST_INJECT = 0x10000
FOS_TEST_STALL = 0x20000

FOS_MAX_LAYERS = 8
FOS_NCOUNT = 6
FOS_MIE_MAX_TERMS = 512

_lock = threading.Lock()
_lib = None


class FosError(RuntimeError):
    def __init__(self, status: int, where: str):
        self.status = status
        extra = ""
        if status in (FOS_ERR_CUDA, FOS_ERR_NOMEM):
            extra = f" [{fos_last_cuda_error()}]"
        super().__init__(f"{where}: {fos_status_string(status)} (status {status}){extra}")


class FosBatch(ctypes.Structure):
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


def _checked() -> bool:
    """FOS_CHECKED=1 selects the checked build (in-kernel index checks in the walk)."""
    return os.environ.get("FOS_CHECKED", "") == "1"


def lib_path() -> str:
    return _build.LIB_CHECKED if _checked() else _build.LIB


def lib():
    """Loads libfos.so (building it first if the sources are newer)."""
    global _lib
    with _lock:
        if _lib is None:
            path = _build.build(checked=_checked())
            if not os.path.exists(path):
                raise RuntimeError("libfos.so is missing: the CUDA path cannot run")
            L = ctypes.CDLL(path)
            vp, i32, i64, u32, u64 = (ctypes.c_void_p, ctypes.c_int, ctypes.c_longlong,
                                      ctypes.c_uint, ctypes.c_ulonglong)
            L.fos_status_string.argtypes = [i32]
            L.fos_status_string.restype = ctypes.c_char_p
            L.fos_api_version.restype = i32
            L.fos_sync_status.argtypes = [vp, i32]
            L.fos_mie_properties.argtypes = ([i32, vp, i32, vp, vp, i32, vp, vp, vp, vp, vp]
                                             + [vp] * 6 + [u32, vp])
            L.fos_mc_spectrum.argtypes = [ctypes.POINTER(FosBatch), vp, vp, i64, u32, vp]
            L.fos_mc_set_tuning.argtypes = [i32, i32]
            L.fos_mc_get_tuning.argtypes = [ctypes.POINTER(FosBatch), u32, ctypes.POINTER(i32),
                                            ctypes.POINTER(i32)]
            L.fos_mc_autotune.argtypes = [ctypes.POINTER(FosBatch), u32, vp,
                                          ctypes.POINTER(i32), ctypes.POINTER(i32)]
            L.fos_mc_walk_times.argtypes = [vp, i32, ctypes.POINTER(i32)]
            L.fos_philox4x32_10.argtypes = [vp, u32, u32, vp, i64, vp]
            L.fos_walk_math_f32.argtypes = [vp, vp, vp, i64, vp]
            L.fos_walk_math_fast_f32.argtypes = [vp, vp, vp, i64, vp]
            for name in ("fos_sync_status", "fos_mie_properties", "fos_mc_spectrum",
                         "fos_mc_set_tuning", "fos_mc_get_tuning", "fos_mc_autotune",
                         "fos_mc_walk_times", "fos_philox4x32_10", "fos_walk_math_f32",
                         "fos_walk_math_fast_f32"):
                getattr(L, name).restype = i32
            _lib = L
    return _lib


def fos_status_string(status: int) -> str:
    return lib().fos_status_string(int(status)).decode()


def fos_last_cuda_error() -> str:
    fn = lib().fos_last_cuda_error
    fn.restype = ctypes.c_char_p
    return (fn() or b"").decode()


def check(status: int, where: str, allow=(FOS_OK,)) -> int:
    if status not in allow:
        raise FosError(status, where)
    return status


def _stream(stream):
    if stream is None:
        return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    if isinstance(stream, torch.cuda.Stream):
        return ctypes.c_void_p(stream.cuda_stream)
    return ctypes.c_void_p(int(stream))


def _dev(t, dtype, name, allow_none=False):
    if t is None:
        if allow_none:
            return None
        raise ValueError(f"{name} is required")
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise ValueError(f"{name} must be a CUDA tensor")
    if t.dtype != dtype:
        raise ValueError(f"{name} must be {dtype}, got {t.dtype}")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")
    return t.data_ptr()


# --------------------------------------------------------------------------- Mie
def fos_mie_properties(wl, nm_re, nm_im, species_group, np_re, np_im, radius, vol_frac,
                       mu_s, mu_a, g, q_ext=None, q_sca=None, g_species=None, flags=0,
                       stream=None) -> int:
    n_wl = wl.numel()
    n_groups = nm_re.numel() // max(n_wl, 1)
    n_species = radius.numel() if radius is not None else 0
    f64, i32 = torch.float64, torch.int32
    args = [n_wl, _dev(wl, f64, "wl"), n_groups, _dev(nm_re, f64, "nm_re"),
            _dev(nm_im, f64, "nm_im"), n_species,
            _dev(species_group, i32, "species_group", n_species == 0),
            _dev(np_re, f64, "np_re", n_species == 0), _dev(np_im, f64, "np_im", n_species == 0),
            _dev(radius, f64, "radius", n_species == 0),
            _dev(vol_frac, f64, "vol_frac", n_species == 0),
            _dev(mu_s, f64, "mu_s"), _dev(mu_a, f64, "mu_a"), _dev(g, f64, "g"),
            _dev(q_ext, f64, "q_ext", True), _dev(q_sca, f64, "q_sca", True),
            _dev(g_species, f64, "g_species", True), int(flags), _stream(stream)]
    return lib().fos_mie_properties(*args)


def fos_mie_properties_cs(wl, nm_re, nm_im, species_group, ns_re, ns_im, nc_re, nc_im,
                          radius, core_radius, vol_frac, mu_s, mu_a, g, q_ext=None, q_sca=None,
                          g_species=None, flags=0, stream=None) -> int:
    n_wl = wl.numel()
    n_groups = nm_re.numel() // max(n_wl, 1)
    n_species = radius.numel() if radius is not None else 0
    f64, i32 = torch.float64, torch.int32
    none = n_species == 0
    args = [n_wl, _dev(wl, f64, "wl"), n_groups, _dev(nm_re, f64, "nm_re"),
            _dev(nm_im, f64, "nm_im"), n_species,
            _dev(species_group, i32, "species_group", none),
            _dev(ns_re, f64, "ns_re", none), _dev(ns_im, f64, "ns_im", none),
            _dev(nc_re, f64, "nc_re", none), _dev(nc_im, f64, "nc_im", none),
            _dev(radius, f64, "radius", none), _dev(core_radius, f64, "core_radius", none),
            _dev(vol_frac, f64, "vol_frac", none),
            _dev(mu_s, f64, "mu_s"), _dev(mu_a, f64, "mu_a"), _dev(g, f64, "g"),
            _dev(q_ext, f64, "q_ext", True), _dev(q_sca, f64, "q_sca", True),
            _dev(g_species, f64, "g_species", True), int(flags), _stream(stream)]
    fn = lib().fos_mie_properties_cs
    fn.argtypes = ([ctypes.c_int, ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p,
                    ctypes.c_int] + [ctypes.c_void_p] * 14 + [ctypes.c_uint, ctypes.c_void_p])
    fn.restype = ctypes.c_int
    return fn(*args)


def fos_size_distribution(diameter: float, sigma: float, vol_frac: float, n: int = 101):
    """(radius [k], vol_frac [k]) NumPy arrays of the sizes a diameter distribution expands to."""
    import numpy as np
    r = np.zeros(max(n, 1))
    f = np.zeros(max(n, 1))
    k = ctypes.c_int(0)
    fn = lib().fos_size_distribution
    fn.argtypes = [ctypes.c_double, ctypes.c_double, ctypes.c_double, ctypes.c_int,
                   ctypes.c_void_p, ctypes.c_void_p, ctypes.POINTER(ctypes.c_int)]
    fn.restype = ctypes.c_int
    check(fn(float(diameter), float(sigma), float(vol_frac), int(n), r.ctypes.data,
             f.ctypes.data, ctypes.byref(k)), "fos_size_distribution")
    return r[: k.value].copy(), f[: k.value].copy()


# --------------------------------------------------------------------------- MC
def make_batch(n_stacks, n_wl, max_layers, mu_s, mu_a, g, n_layer, thickness,
               n_layers=None, n_above=None, n_below=None, substrate_R=None, n_photons=None,
               photons_per_item=0, photon_first=None, item_list=None, seed=0,
               item_id_base=0, max_events=0, cos_incidence=None, k_below=None) -> FosBatch:
    """Fills the C struct from CUDA tensors.  The struct keeps references to the tensors,
    so temporaries passed here stay allocated as long as the struct lives."""
    f64, i32, i64 = torch.float64, torch.int32, torch.int64
    b = FosBatch()
    b._keep = [t for t in (mu_s, mu_a, g, n_layer, thickness, n_layers, n_above, n_below,
                           substrate_R, n_photons, photon_first, item_list, cos_incidence,
                           k_below) if t is not None]
    b.n_stacks, b.n_wl, b.max_layers = int(n_stacks), int(n_wl), int(max_layers)
    b.n_layers = _dev(n_layers, i32, "n_layers", True)
    b.mu_s = _dev(mu_s, f64, "mu_s")
    b.mu_a = _dev(mu_a, f64, "mu_a")
    b.g = _dev(g, f64, "g")
    b.n_layer = _dev(n_layer, f64, "n_layer")
    b.thickness = _dev(thickness, f64, "thickness")
    b.n_above = _dev(n_above, f64, "n_above", True)
    b.n_below = _dev(n_below, f64, "n_below", True)
    b.substrate_R = _dev(substrate_R, f64, "substrate_R", True)
    b.n_photons = _dev(n_photons, i64, "n_photons", True)
    b.photons_per_item = int(photons_per_item)
    b.photon_first = _dev(photon_first, i64, "photon_first", True)
    b.item_list = _dev(item_list, i32, "item_list", True)
    b.n_list = int(item_list.numel()) if item_list is not None else 0
    b.seed = int(seed) & 0xFFFFFFFFFFFFFFFF
    b.item_id_base = int(item_id_base) & 0xFFFFFFFF
    b.max_events = int(max_events)
    b.cos_incidence = _dev(cos_incidence, f64, "cos_incidence", True)
    b.k_below = _dev(k_below, f64, "k_below", True)
    return b


def fos_mc_spectrum(batch: FosBatch, counts, photon_log=None, log_stride=0, flags=0,
                    stream=None) -> int:
    return lib().fos_mc_spectrum(ctypes.byref(batch), _dev(counts, torch.int64, "counts"),
                                 _dev(photon_log, torch.int32, "photon_log", True),
                                 int(log_stride), int(flags), _stream(stream))


def fos_solar_weighted(n_stacks: int, wl, G, counts, out, flags=0, stream=None) -> int:
    fn = lib().fos_solar_weighted
    fn.argtypes = [ctypes.c_int, ctypes.c_int] + [ctypes.c_void_p] * 4 + [ctypes.c_uint,
                                                                           ctypes.c_void_p]
    fn.restype = ctypes.c_int
    return fn(int(n_stacks), int(wl.numel()), _dev(wl, torch.float64, "wl"),
              _dev(G, torch.float64, "G"), _dev(counts, torch.int64, "counts"),
              _dev(out, torch.float64, "out"), int(flags), _stream(stream))


def fos_mc_set_tuning(block: int, photons_per_thread: int) -> int:
    return lib().fos_mc_set_tuning(int(block), int(photons_per_thread))


def fos_mc_get_tuning(batch: FosBatch, flags: int = 0):
    b, p = ctypes.c_int(), ctypes.c_int()
    check(lib().fos_mc_get_tuning(ctypes.byref(batch), int(flags), ctypes.byref(b),
                                  ctypes.byref(p)), "fos_mc_get_tuning")
    return b.value, p.value


def fos_mc_autotune(batch: FosBatch, flags: int = 0, stream=None):
    b, p = ctypes.c_int(), ctypes.c_int()
    check(lib().fos_mc_autotune(ctypes.byref(batch), int(flags), _stream(stream),
                                ctypes.byref(b), ctypes.byref(p)), "fos_mc_autotune")
    return b.value, p.value


def fos_mc_walk_times():
    """Per-block (start, end) ns of the last walk run with FOS_RECORD_TIMES (host int64
    array [n_blocks, 2]; empty if none)."""
    import numpy as np
    n = ctypes.c_int()
    check(lib().fos_mc_walk_times(None, 0, ctypes.byref(n)), "fos_mc_walk_times")
    out = np.zeros((max(n.value, 1), 2), np.int64)
    if n.value:
        check(lib().fos_mc_walk_times(out.ctypes.data, n.value, ctypes.byref(n)),
              "fos_mc_walk_times")
    return out[: n.value]


def fos_sync_status(stream=None, timeout_ms: int = 0) -> int:
    return lib().fos_sync_status(_stream(stream), int(timeout_ms))


# --------------------------------------------------------------------------- diagnostics
def fos_philox4x32_10(ctr, k0: int, k1: int, out, stream=None, curand: bool = False) -> int:
    n = ctr.numel() // 4
    fn = (_sfn("fos_philox4x32_10_curand", [ctypes.c_void_p, ctypes.c_uint, ctypes.c_uint,
                                            ctypes.c_void_p, ctypes.c_longlong, ctypes.c_void_p])
          if curand else lib().fos_philox4x32_10)
    return fn(_dev(ctr, torch.int32, "ctr"), int(k0) & 0xFFFFFFFF, int(k1) & 0xFFFFFFFF,
              _dev(out, torch.int32, "out"), n, _stream(stream))


def fos_walk_math_f32(u, neg_log=None, cos2pi=None, stream=None, fast: bool = False) -> int:
    f32 = torch.float32
    fn = lib().fos_walk_math_fast_f32 if fast else lib().fos_walk_math_f32
    return fn(_dev(u, f32, "u"), _dev(neg_log, f32, "neg_log", True),
              _dev(cos2pi, f32, "cos2pi", True), u.numel(), _stream(stream))


# --------------------------------------------------------------------------- surrogate
_SFN = {}


def _sfn(name, argtypes, restype=ctypes.c_int):
    """The library function `name`, its ctypes signature set once."""
    fn = _SFN.get(name)
    if fn is None:
        fn = getattr(lib(), name)
        fn.argtypes = argtypes
        fn.restype = restype
        _SFN[name] = fn
    return fn


def fos_surrogate_model_bytes() -> int:
    return int(_sfn("fos_surrogate_model_bytes", [], ctypes.c_size_t)())


def fos_surrogate_param_count() -> int:
    return int(_sfn("fos_surrogate_param_count", [], ctypes.c_longlong)())


def fos_surrogate_param_offsets():
    w = (ctypes.c_longlong * 5)()
    b = (ctypes.c_longlong * 5)()
    check(_sfn("fos_surrogate_param_offsets", [ctypes.c_void_p, ctypes.c_void_p])(w, b),
          "fos_surrogate_param_offsets")
    return list(w), list(b)


def fos_surrogate_init(model, n_members, seed, feat_stats, stream=None) -> int:
    """feat_stats: host sequence of 64 floats (mean[16] | std[16] | lo[16] | hi[16])."""
    st = (ctypes.c_float * 64)(*[float(v) for v in feat_stats])
    return _sfn("fos_surrogate_init", [ctypes.c_void_p, ctypes.c_int, ctypes.c_ulonglong,
                                       ctypes.c_void_p, ctypes.c_void_p])(
        _dev(model, torch.uint8, "model"), int(n_members), int(seed) & 0xFFFFFFFFFFFFFFFF,
        st, _stream(stream))


def fos_surrogate_load(model, member, theta, feat_stats, stream=None) -> int:
    """theta: device float32 [fos_surrogate_param_count()]; feat_stats: 64 host floats."""
    st = (ctypes.c_float * 64)(*[float(v) for v in feat_stats])
    return _sfn("fos_surrogate_load", [ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p,
                                       ctypes.c_void_p, ctypes.c_void_p])(
        _dev(model, torch.uint8, "model"), int(member), _dev(theta, torch.float32, "theta"),
        st, _stream(stream))


def fos_surrogate_features_slab(n_layer, mu_s, mu_a, g, thickness, features, flags=0,
                                stream=None) -> int:
    f64 = torch.float64
    return _sfn("fos_surrogate_features_slab", [ctypes.c_longlong] + [ctypes.c_void_p] * 6 +
                [ctypes.c_uint, ctypes.c_void_p])(
        int(n_layer.numel()), _dev(n_layer, f64, "n_layer"), _dev(mu_s, f64, "mu_s"),
        _dev(mu_a, f64, "mu_a"), _dev(g, f64, "g"), _dev(thickness, f64, "thickness"),
        _dev(features, torch.float32, "features"), int(flags), _stream(stream))


def fos_surrogate_features(wl, np_re, np_im, radius, vol_frac, thickness, g, mu_s, mu_a,
                           features, flags=0, stream=None) -> int:
    f64 = torch.float64
    n_designs, n_wl = radius.numel(), wl.numel()
    return _sfn("fos_surrogate_features", [ctypes.c_int, ctypes.c_int] + [ctypes.c_void_p] * 10
                + [ctypes.c_uint, ctypes.c_void_p])(
        n_designs, n_wl, _dev(wl, f64, "wl"), _dev(np_re, f64, "np_re"),
        _dev(np_im, f64, "np_im"), _dev(radius, f64, "radius"), _dev(vol_frac, f64, "vol_frac"),
        _dev(thickness, f64, "thickness"), _dev(g, f64, "g"), _dev(mu_s, f64, "mu_s"),
        _dev(mu_a, f64, "mu_a"), _dev(features, torch.float32, "features"), int(flags),
        _stream(stream))


def fos_surrogate_feature_stats(features, stats, stream=None) -> int:
    return _sfn("fos_surrogate_feature_stats", [ctypes.c_void_p, ctypes.c_longlong,
                                                ctypes.c_void_p, ctypes.c_void_p])(
        _dev(features, torch.float32, "features"), features.numel() // 9,
        _dev(stats, torch.float32, "stats"), _stream(stream))


def fos_counts_to_fractions(counts, fractions, rows=None, stream=None) -> int:
    n = counts.numel() // FOS_NCOUNT
    return _sfn("fos_counts_to_fractions", [ctypes.c_void_p, ctypes.c_longlong, ctypes.c_void_p,
                                            ctypes.c_void_p, ctypes.c_void_p])(
        _dev(counts, torch.int64, "counts"), n, _dev(rows, torch.int32, "rows", True),
        _dev(fractions, torch.float32, "fractions"), _stream(stream))


def fos_mask_to_rows(mask, rows, count, stream=None) -> int:
    return _sfn("fos_mask_to_rows", [ctypes.c_void_p, ctypes.c_longlong, ctypes.c_void_p,
                                     ctypes.c_void_p, ctypes.c_void_p])(
        _dev(mask, torch.uint8, "mask"), mask.numel(), _dev(rows, torch.int32, "rows"),
        _dev(count, torch.int64, "count"), _stream(stream))


def fos_surrogate_fit(model, n_members, features, targets, batch, seed, n_steps, lr_max,
                      lr_min, schedule_origin, schedule_total, loss_out=None, flags=0,
                      stream=None) -> int:
    f32 = torch.float32
    n_rows = features.numel() // 9
    return _sfn("fos_surrogate_fit",
                [ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p,
                 ctypes.c_longlong, ctypes.c_int, ctypes.c_ulonglong, ctypes.c_int,
                 ctypes.c_float, ctypes.c_float, ctypes.c_int, ctypes.c_int, ctypes.c_void_p,
                 ctypes.c_uint, ctypes.c_void_p])(
        _dev(model, torch.uint8, "model"), int(n_members), _dev(features, f32, "features"),
        _dev(targets, f32, "targets"), n_rows, int(batch), int(seed) & 0xFFFFFFFFFFFFFFFF,
        int(n_steps), float(lr_max), float(lr_min), int(schedule_origin), int(schedule_total),
        _dev(loss_out, f32, "loss_out", True), int(flags), _stream(stream))


def fos_surrogate_train_step(model, member, features, targets, batch, seed, step, lr,
                             batch_rows=None, loss_out=None, grad_out=None, flags=0,
                             stream=None) -> int:
    f32 = torch.float32
    n_rows = features.numel() // 9
    return _sfn("fos_surrogate_train_step",
                [ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_longlong,
                 ctypes.c_int, ctypes.c_void_p, ctypes.c_ulonglong, ctypes.c_int, ctypes.c_float,
                 ctypes.c_void_p, ctypes.c_void_p, ctypes.c_uint, ctypes.c_void_p])(
        _dev(model, torch.uint8, "model"), int(member), _dev(features, f32, "features"),
        _dev(targets, f32, "targets"), n_rows, int(batch),
        _dev(batch_rows, torch.int32, "batch_rows", True), int(seed) & 0xFFFFFFFFFFFFFFFF,
        int(step), float(lr), _dev(loss_out, f32, "loss_out", True),
        _dev(grad_out, f32, "grad_out", True), int(flags), _stream(stream))


def fos_surrogate_predict(model, n_members, features, rat, spread=None, needs_mc=None,
                          threshold=0.01, flags=0, stream=None) -> int:
    f32 = torch.float32
    n_rows = features.numel() // 9
    return _sfn("fos_surrogate_predict",
                [ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p, ctypes.c_longlong, ctypes.c_void_p,
                 ctypes.c_void_p, ctypes.c_void_p, ctypes.c_float, ctypes.c_uint, ctypes.c_void_p])(
        _dev(model, torch.uint8, "model"), int(n_members), _dev(features, f32, "features"), n_rows,
        _dev(rat, f32, "rat"), _dev(spread, f32, "spread", True),
        _dev(needs_mc, torch.uint8, "needs_mc", True), float(threshold), int(flags),
        _stream(stream))


def fos_gemm_bf16(A, B, C, splits=1, flags=0, stream=None) -> int:
    M, K = A.shape
    N = B.shape[0]
    return _sfn("fos_gemm_bf16", [ctypes.c_void_p] * 3 + [ctypes.c_int] * 4
                + [ctypes.c_uint, ctypes.c_void_p])(
        _dev(A, torch.bfloat16, "A"), _dev(B, torch.bfloat16, "B"), _dev(C, torch.float32, "C"),
        int(M), int(N), int(K), int(splits), int(flags), _stream(stream))


# --------------------------------------------------------------------------- no allocation
def fos_mc_spectrum_noalloc(batch: FosBatch, counts, flags=0, stream=None) -> int:
    """fos_mc_spectrum for callers that cannot allocate device memory (scratch is a
    fixed static device array of the library; at most FOS_NOALLOC_MAX_ITEMS items)."""
    L = lib()
    fn = L.fos_mc_spectrum_noalloc
    fn.argtypes = [ctypes.POINTER(FosBatch), ctypes.c_void_p, ctypes.c_uint, ctypes.c_void_p]
    fn.restype = ctypes.c_int
    return fn(ctypes.byref(batch), _dev(counts, torch.int64, "counts"), int(flags),
              _stream(stream))


FOS_NOALLOC_MAX_ITEMS = 4096
