"""Shared helpers of the GPU tests: run the C-ABI on batches given as NumPy dicts."""
from __future__ import annotations

import numpy as np
import torch

from paper_2409_00165_gb300 import fos


def to_dev(a, dtype):
    if a is None:
        return None
    return torch.as_tensor(np.ascontiguousarray(a), dtype=dtype, device="cuda")


def gpu_mc(batch: dict, photon_log: bool = False, flags: int = 0, allow=(fos.FOS_OK,)):
    """Runs fos_mc_spectrum on a batch dict (the oracle's format)."""
    f64, i32, i64 = torch.float64, torch.int32, torch.int64
    keep = dict(
        n_layers=to_dev(batch.get("n_layers"), i32),
        mu_s=to_dev(batch["mu_s"], f64), mu_a=to_dev(batch["mu_a"], f64),
        g=to_dev(batch["g"], f64), n_layer=to_dev(batch["n_layer"], f64),
        thickness=to_dev(batch["thickness"], f64),
        n_above=to_dev(batch.get("n_above"), f64), n_below=to_dev(batch.get("n_below"), f64),
        substrate_R=to_dev(batch.get("substrate_R"), f64),
        n_photons=to_dev(batch.get("n_photons"), i64),
        photon_first=to_dev(batch.get("photon_first"), i64),
        item_list=to_dev(batch.get("item_list"), i32),
        cos_incidence=to_dev(batch.get("cos_incidence"), f64),
        k_below=to_dev(batch.get("k_below"), f64),
    )
    b = fos.make_batch(batch["n_stacks"], batch["n_wl"], batch["max_layers"],
                       photons_per_item=int(batch.get("photons_per_item", 0)),
                       seed=int(batch.get("seed", 0)),
                       item_id_base=int(batch.get("item_id_base", 0)),
                       max_events=int(batch.get("max_events", 0)), **keep)
    n_items = int(batch["n_stacks"]) * int(batch["n_wl"])
    n_run = len(batch["item_list"]) if batch.get("item_list") is not None else n_items
    counts = torch.full((max(n_run, 1), fos.FOS_NCOUNT), -1, dtype=i64, device="cuda")
    log = None
    stride = 0
    if photon_log:
        if batch.get("n_photons") is not None:
            stride = int(np.max(batch["n_photons"]))
        else:
            stride = int(batch["photons_per_item"])
        log = torch.full((max(n_run, 1), max(stride, 1)), -1, dtype=i32, device="cuda")
    st = fos.fos_mc_spectrum(b, counts, log, stride, flags)
    torch.cuda.synchronize()
    fos.check(st, "fos_mc_spectrum", allow)
    c = counts.cpu().numpy()[:n_run]
    if photon_log:
        return c, log.cpu().numpy()[:n_run], st
    return c, st


def mie_inputs_to_dev(m: dict):
    nm = np.asarray(m["nm"], np.complex128)
    n_p = np.asarray(m["n_p"], np.complex128)
    f64 = torch.float64
    out = dict(
        wl=to_dev(m["wl"], f64),
        nm_re=to_dev(nm.real.reshape(-1), f64), nm_im=to_dev(nm.imag.reshape(-1), f64),
        species_group=to_dev(m["species_group"], torch.int32),
        np_re=to_dev(n_p.real.reshape(-1), f64), np_im=to_dev(n_p.imag.reshape(-1), f64),
        radius=to_dev(m["radius"], f64), vol_frac=to_dev(m["vol_frac"], f64))
    if "core_radius" in m:
        nc = np.asarray(m["n_core"], np.complex128)
        out.update(core_radius=to_dev(m["core_radius"], f64),
                   nc_re=to_dev(nc.real.reshape(-1), f64), nc_im=to_dev(nc.imag.reshape(-1), f64))
    return out


def gpu_mie(m: dict, allow=(fos.FOS_OK,), flags: int = 0):
    d = mie_inputs_to_dev(m)
    n_wl = len(m["wl"])
    n_groups = np.asarray(m["nm"]).shape[0]
    n_species = len(m["radius"])
    f64 = torch.float64
    out = {k: torch.zeros(n_groups * n_wl, dtype=f64, device="cuda") for k in ("mu_s", "mu_a", "g")}
    q = {k: torch.zeros(max(n_species * n_wl, 1), dtype=f64, device="cuda")
         for k in ("q_ext", "q_sca", "g_species")}
    if "core_radius" in m:
        name = "fos_mie_properties_cs"
        st = fos.fos_mie_properties_cs(d["wl"], d["nm_re"], d["nm_im"], d["species_group"],
                                       d["np_re"], d["np_im"], d["nc_re"], d["nc_im"],
                                       d["radius"], d["core_radius"], d["vol_frac"], out["mu_s"],
                                       out["mu_a"], out["g"], q["q_ext"], q["q_sca"],
                                       q["g_species"], flags=flags)
    else:
        name = "fos_mie_properties"
        st = fos.fos_mie_properties(d["wl"], d["nm_re"], d["nm_im"], d["species_group"],
                                    d["np_re"], d["np_im"], d["radius"], d["vol_frac"],
                                    out["mu_s"], out["mu_a"], out["g"], q["q_ext"], q["q_sca"],
                                    q["g_species"], flags=flags)
    torch.cuda.synchronize()
    fos.check(st, name, allow)
    res = {k: v.cpu().numpy().reshape(n_groups, n_wl) for k, v in out.items()}
    res.update({k: v.cpu().numpy()[: n_species * n_wl].reshape(n_species, n_wl)
                for k, v in q.items()})
    res["status"] = st
    return res


def mc_batch_from_media(m: dict, props: dict, photons=None) -> dict:
    """MC batch dict from a media description and per-group optical properties."""
    n_wl = len(m["wl"])
    nm = np.asarray(m["nm"])
    b = dict(n_stacks=m["n_stacks"], n_wl=n_wl, max_layers=m["max_layers"],
             n_layers=m["n_layers"], mu_s=props["mu_s"].reshape(-1),
             mu_a=props["mu_a"].reshape(-1), g=props["g"].reshape(-1),
             n_layer=nm.real.reshape(-1), thickness=m["thickness"],
             substrate_R=m.get("substrate_R"), n_photons=m.get("n_photons"),
             photons_per_item=m.get("photons_per_item", 0), seed=m.get("seed", 1))
    if photons is not None:
        b["n_photons"] = None
        b["photons_per_item"] = int(photons)
    return b
