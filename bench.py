#!/usr/bin/env python
"""Benchmark of the FOS hot path on GB300: FP64 Mie + FP32 Monte Carlo photon transport.

One step = one full-spectrum paint layer (400 wavelengths 0.3-2.5 um, spheres r = 0.2 um
at volume fraction 0.10 in a 300 um layer of n = 1.48 + 1e-5 lambda i, particle n =
2.5 + 0.05/lambda^2 with k = 0.5 below 0.4 um and 1e-4 above, air both sides, 1e6
photons per wavelength): fos_mie_properties then fos_mc_spectrum.  The metric is
photon-steps/s (collision events per second, from the kernel's own tallies); spectra/s
is reported beside it.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl fos|reference]

Under torchrun every rank runs its own spectrum (independent photons: weak scaling,
no collective on the data path); rank 0 prints one JSON line.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = ("photon-steps/s and spectra/s (MC vs surrogate, same GB300, "
          "≤0.01 abs R/A/T error)")
UNIT = "photon-steps/s"
WORKLOAD = ("paint layer: 400 wavelengths 0.3-2.5 um; r = 0.2 um, f = 0.10, 300 um; "
            "Cauchy particle n = 2.5+0.05/lambda^2, k = 0.5 (<0.4 um) / 1e-4; "
            "matrix n = 1.48, k = 1e-5 lambda; 1e6 photons per wavelength; FP64 Mie + FP32 MC")

# Algorithmic FP32/INT operations of one collision event of the walk (hand tally of the
# operations the method performs, each IEEE +,-,*,/,sqrt,fma, compare, select, integer
# multiply, logic op or conversion counted once):
#   Philox4x32-10: 10 rounds x (2 mul.hi + 2 mul.lo + 2 three-input xor) + 18 key adds = 78
#   4 uniforms: 4 x (shift/or 2 + convert 1 + scale 1) = 16
#   -ln u series: 22;  free-path/boundary test and move: 11;  absorption test: 1
#   Henyey-Greenstein inversion: 9;  direction update incl. cos(2 pi u) series: 24;  counters: 1
OPS_PER_STEP = 78 + 16 + 22 + 11 + 1 + 9 + 24 + 1   # = 162


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["fos", "reference"], default="fos")
    ap.add_argument("--photons", type=int, default=1000000)
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--cpu-seconds", type=float, default=15.0)
    ap.add_argument("--no-autotune", action="store_true")
    ap.add_argument("--surrogate", choices=["full", "quick", "off"], default="full",
                    help="surrogate leg (1 GPU only): MC training data, ensemble training, "
                         "design sweep with MC fallback and audit")
    ap.add_argument("--stacks", action="store_true",
                    help="also time the uneven multilayer-stack batch once")
    ap.add_argument("--legs", choices=["on", "off"], default="on",
                    help="workload legs after the timed steps (1 GPU only): size "
                         "distributions, core-shell spheres, oblique incidence on a conductor")
    return ap.parse_args()


# ------------------------------------------------------------------------ CPU (oracle)
def _oracle_props(m):
    import oracle
    return oracle.mie_properties(m["wl"], m["nm"], m["species_group"], m["n_p"], m["radius"],
                                 m["vol_frac"])


def oracle_sample(m, props, photons_per_wl: int, n_threads: int, wl_idx):
    """Runs the oracle walk (FP32 mirror) on a sample of wavelengths, threads sharing
    photon ranges; returns (collisions, photons, seconds)."""
    import numpy as np

    import oracle
    from concurrent.futures import ThreadPoolExecutor
    n_wl = m["n_wl"]
    base = dict(n_stacks=1, n_wl=n_wl, max_layers=1, mu_s=props["mu_s"].reshape(-1),
                mu_a=props["mu_a"].reshape(-1), g=props["g"].reshape(-1),
                n_layer=m["nm"].real.reshape(-1), thickness=m["thickness"], seed=m["seed"],
                item_list=np.asarray(wl_idx, np.int32))
    shards = []
    per = photons_per_wl // n_threads
    for t in range(n_threads):
        b = dict(base)
        cnt = per if t < n_threads - 1 else photons_per_wl - per * (n_threads - 1)
        b["photons_per_item"] = cnt
        b["photon_first"] = np.full(n_wl, t * per, np.int64)
        shards.append(b)
    t0 = time.perf_counter()
    with ThreadPoolExecutor(max_workers=n_threads) as ex:
        res = list(ex.map(lambda b: oracle.mc_run(b, fp32=True), shards))
    dt = time.perf_counter() - t0
    tot = sum(r.sum(axis=0) for r in res)
    return int(tot[4]), int(photons_per_wl * len(wl_idx)), dt


def cpu_baseline(m, seconds: float):
    import numpy as np
    props = _oracle_props(m)
    cores = os.cpu_count() or 1
    wl_idx = np.linspace(0, m["n_wl"] - 1, 8).round().astype(int)
    # calibrate on a small run, then size the sample for ~`seconds` of wall time
    c0, p0, t0 = oracle_sample(m, props, 64 * cores, cores, wl_idx)
    per_photon = t0 / max(p0, 1)
    n = int(max(64 * cores, min(m["photons_per_item"], seconds / max(per_photon, 1e-9) / 8)))
    coll, phot, dt = oracle_sample(m, props, n, cores, wl_idx)
    return dict(value=coll / dt, unit=UNIT, cores=cores, kind="oracle",
                sample=f"8 of 400 wavelengths (evenly spaced) x {n} photons each, FP32-mirror "
                       f"oracle walk, {cores} host threads sharing photon ranges; "
                       f"{coll} photon-steps in {dt:.1f} s",
                photons_per_s=phot / dt)


# ------------------------------------------------------------------------ clocks
class ClockSampler:
    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.path = None

    def __enter__(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
                 "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
                 "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.index}", f"--query-gpu={q}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *a):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        if not self.path or not os.path.exists(self.path):
            return None
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx.append(float(f[2]))
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        os.unlink(self.path)
        if not sm:
            return None
        return dict(sm_mhz=statistics.median(sm), sm_max_mhz=max(mx), reasons=sorted(reasons),
                    samples=len(sm))


# ------------------------------------------------------------------------ GPU arm
def run_fos(args):
    import numpy as np
    import torch
    import torch.distributed as dist

    from paper_2409_00165_gb300 import fos
    from paper_2409_00165_gb300 import workloads as W

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    dev = torch.device("cuda", local)
    fos.lib()

    m = W.paint_layer(photons=args.photons)
    f64, i64 = torch.float64, torch.int64
    host = dict(wl=torch.as_tensor(m["wl"], dtype=f64),
                **{k: torch.as_tensor(v, dtype=f64) for k, v in W.media_arrays(m).items()},
                sg=torch.as_tensor(m["species_group"], dtype=torch.int32),
                radius=torch.as_tensor(m["radius"], dtype=f64),
                vol_frac=torch.as_tensor(m["vol_frac"], dtype=f64),
                thickness=torch.as_tensor(m["thickness"], dtype=f64),
                G=torch.as_tensor(W.solar_like_irradiance(m["wl"]), dtype=f64))
    d = {k: v.to(dev) for k, v in host.items()}
    n_wl = m["n_wl"]
    mu_s, mu_a, g = (torch.zeros(n_wl, dtype=f64, device=dev) for _ in range(3))
    counts = torch.zeros((n_wl, fos.FOS_NCOUNT), dtype=i64, device=dev)
    solar = torch.zeros(3, dtype=f64, device=dev)   # Eq. 21 R_s, A_s, T_s
    stream = torch.cuda.current_stream()
    l2 = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)

    def step(seed, flags=fos.FOS_ASYNC, ev=None, src=d):
        fos.check(fos.fos_mie_properties(src["wl"], src["nm_re"], src["nm_im"], src["sg"],
                                         src["np_re"], src["np_im"], src["radius"],
                                         src["vol_frac"], mu_s, mu_a, g, flags=flags),
                  "fos_mie_properties")
        b = fos.make_batch(1, n_wl, 1, mu_s, mu_a, g, src["nm_re"], src["thickness"],
                           photons_per_item=m["photons_per_item"], seed=seed,
                           item_id_base=rank * n_wl)
        if ev is not None:
            ev[0].record(stream)
        fos.check(fos.fos_mc_spectrum(b, counts, None, 0, flags), "fos_mc_spectrum")
        if ev is not None:
            ev[1].record(stream)
        fos.check(fos.fos_solar_weighted(1, src["wl"], src["G"], counts, solar,
                                         flags=flags & fos.FOS_ASYNC), "fos_solar_weighted")
        return b

    # first call tunes the launch shape for this batch (synchronous, untimed)
    b0 = step(1000, flags=0 if args.no_autotune else fos.FOS_AUTOTUNE)
    tuning = fos.fos_mc_get_tuning(b0)
    for w in range(args.warmup):
        step(1001 + w)
    fos.check(fos.fos_sync_status(stream), "warmup")
    torch.cuda.synchronize()

    K = args.steps
    per_step_counts = torch.zeros((K, n_wl, fos.FOS_NCOUNT), dtype=i64, device=dev)
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
           for _ in range(K)]
    t_start, t_end = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    with ClockSampler(local) as clk:
        t_start.record(stream)
        for k in range(K):
            l2.fill_(float(k))                   # flush L2 between steps (timed)
            step(2000 + k, ev=evs[k])
            per_step_counts[k].copy_(counts)
        t_end.record(stream)
        torch.cuda.synchronize()
    st = fos.fos_sync_status(stream)
    fos.check(st, "timed steps")
    if world > 1:
        dist.barrier()
    ms_total = t_start.elapsed_time(t_end)
    walk_ms = [a.elapsed_time(b) for a, b in evs]
    pc = per_step_counts.cpu().numpy()
    coll = int(pc[:, :, 4].sum())
    photons = int(pc[:, :, :4].sum())
    assert photons == K * n_wl * m["photons_per_item"], "photon conservation failed"
    local_vals = torch.tensor([ms_total, float(coll), float(photons)], dtype=torch.float64,
                              device=dev)
    if world > 1:
        mx = local_vals.clone()
        dist.all_reduce(mx, op=dist.ReduceOp.MAX)
        sm = local_vals.clone()
        dist.all_reduce(sm, op=dist.ReduceOp.SUM)
        ms_total, coll_all, phot_all = mx[0].item(), sm[1].item(), sm[2].item()
    else:
        coll_all, phot_all = float(coll), float(photons)
    secs = ms_total / 1e3
    value = coll_all / secs
    spectra_per_s = world * K / secs

    # e2e: the same step from pinned host buffers, copies and the count read-back timed
    e2e = None
    if not args.no_e2e:
        pinned = {k: v.pin_memory() for k, v in host.items()}
        counts_h = torch.empty((n_wl, fos.FOS_NCOUNT), dtype=i64).pin_memory()
        solar_h = torch.empty(3, dtype=f64).pin_memory()
        dd = {k: torch.empty_like(v, device=dev) for k, v in host.items()}
        h2d = sum(v.numel() * v.element_size() for v in pinned.values())
        d2h = counts_h.numel() * counts_h.element_size() + solar_h.numel() * 8
        Ke = max(1, min(K, 3))
        coll_e = 0
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for k in range(Ke):
            for kk, v in pinned.items():
                dd[kk].copy_(v, non_blocking=True)
            step(3000 + k, flags=0, src=dd)
            counts_h.copy_(counts, non_blocking=True)
            solar_h.copy_(solar, non_blocking=True)
            torch.cuda.synchronize()
            coll_e += int(counts_h[:, 4].sum())
        dt = time.perf_counter() - t0
        tot = torch.tensor([dt, float(coll_e)], dtype=torch.float64, device=dev)
        if world > 1:
            mx = tot.clone()
            dist.all_reduce(mx, op=dist.ReduceOp.MAX)
            sm2 = tot.clone()
            dist.all_reduce(sm2, op=dist.ReduceOp.SUM)
            dt, coll_e = mx[0].item(), sm2[1].item()
        e2e = dict(value=coll_e / dt, unit=UNIT, h2d_bytes_per_step=int(h2d),
                   d2h_bytes_per_step=int(d2h), steps=Ke,
                   spectra_per_s=world * Ke / dt)

    if rank != 0:
        if world > 1:
            dist.destroy_process_group()
        return
    clocks = clk.summary()
    walk_s = statistics.mean(walk_ms) / 1e3
    steps_per_launch = coll / K
    achieved = OPS_PER_STEP * steps_per_launch / walk_s / 1e12
    peaks = {}
    try:
        peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        pass
    sm_count = torch.cuda.get_device_properties(dev).multi_processor_count
    f_max = float(peaks.get("sm_max_mhz", 2070.0)) * 1e6
    peak = sm_count * 128 * f_max / 1e12
    roof = dict(bound="alu", achieved=achieved, peak=peak, unit="Top/s", frac=achieved / peak,
                traffic=None,
                kernel="walk_kernel", ops_per_photon_step=OPS_PER_STEP,
                photon_steps_per_launch=steps_per_launch, launch_ms=walk_s * 1e3,
                peak_basis=f"{sm_count} SMs x 128 FP32/INT lanes x {f_max/1e6:.0f} MHz "
                           "(maximum SM clock)")
    if clocks:
        roof["frac_at_sampled_clock"] = achieved / (sm_count * 128 * clocks["sm_mhz"] * 1e6 / 1e12)
    surr = None
    if args.surrogate != "off" and world == 1:
        try:
            surr = run_surrogate(args.surrogate)
        except Exception as exc:  # the surrogate leg must not hide the MC number
            surr = dict(error=str(exc))
    t1 = None
    if args.surrogate != "off" and world == 1:
        try:
            t1 = run_table1(args.surrogate)
        except Exception as exc:
            t1 = dict(error=str(exc))
    stacks = None
    if args.stacks and world == 1:
        stacks = run_stacks()
    dists = cs = bnd = None
    if world == 1 and args.legs == "on":
        try:
            dists = run_distributions()
        except Exception as exc:
            dists = dict(error=str(exc))
        try:
            cs = run_core_shell()
        except Exception as exc:
            cs = dict(error=str(exc))
        try:
            bnd = run_boundaries()
        except Exception as exc:
            bnd = dict(error=str(exc))
    cpu = None
    if not args.no_cpu and world == 1:
        try:
            cpu = cpu_baseline(m, args.cpu_seconds)
        except Exception as exc:  # the baseline must not hide the GPU number
            cpu = dict(error=str(exc))
    line = dict(
        metric=METRIC, value=value, unit=UNIT, n_gpus=world, steps=K, warmup=args.warmup,
        ms_per_step=ms_total / K, higher_is_better=True, scaling="weak", vs_baseline=None,
        dtype="f32", data="synthetic",
        config=dict(workload=WORKLOAD, photons_per_step=n_wl * m["photons_per_item"],
                    wavelengths=n_wl, l2="flushed before every step by a 512 MiB write "
                    "inside the timed region", tuning=dict(block=tuning[0], ppt=tuning[1]),
                    precision="Mie f64, walk f32, tallies int64", parallelism=f"replicas x{world}"),
        spectra_per_s=spectra_per_s, photons_per_s=phot_all / secs,
        photon_steps_per_photon=coll / max(photons, 1),
        e2e=e2e, roofline=roof, cpu_baseline=cpu, clocks=clocks, surrogate=surr,
        layer_stacks=stacks, size_distributions=dists, core_shell=cs,
        oblique_conductor=bnd, table1_network=t1,
        solar_weighted=dict(zip(("R_s", "A_s", "T_s"), solar.cpu().tolist())),
        gpu_launches=6 * K,
        gpu_launches_detail="per step: mie_kernel, emt_kernel, pack_kernel, unit_scan_kernel, "
                            "walk_kernel, solar_kernel",
    )
    print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


# ------------------------------------------------------------------------ surrogate leg
def run_surrogate(mode: str):
    """Surrogate spectra/s vs plain GPU Monte Carlo spectra/s on the same designs.

    Training data: single-layer designs (r, f, d in the workload ranges) x 50 random
    wavelengths per block, Monte Carlo fractions at 3e4 photons; 4 members trained by
    Adam.  Sweep: 1e5 designs x 300 wavelengths, ensemble spread > 0.01 or out-of-range
    rows re-run by Monte Carlo at 1e5 photons; 1 % of rows (0.1 % in quick mode) audited
    by Monte Carlo at 1e5 photons."""
    import torch

    from paper_2409_00165_gb300 import surrogate as S
    cfg = dict(full=dict(designs=20000, blocks=20, wl=50, photons=30000, steps=30000,
                         sweep=100000),
               quick=dict(designs=4000, blocks=10, wl=24, photons=10000, steps=2500,
                          sweep=20000))[mode]
    t0 = time.perf_counter()
    f, y, info = S.training_set(cfg["designs"], cfg["wl"], cfg["blocks"], cfg["photons"], seed=4,
                                log_share=0.5)
    sur = S.Surrogate(4, S.Surrogate.stats_of(f), seed=7)
    t1 = time.perf_counter()
    hist = sur.fit(f, y, steps=cfg["steps"], batch=8192, lr=2e-3, log_every=cfg["steps"] - 1)
    torch.cuda.synchronize()
    t2 = time.perf_counter()
    r = S.sweep(sur, n_designs=cfg["sweep"], n_wl=300, seed=5, threshold=0.01,
                audit_frac=0.01 if mode == "full" else 0.001)
    peaks = {}
    try:
        peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        pass
    peak = float(peaks.get("bf16_tflops", 1900.0))
    r["roofline"] = dict(bound="tensor", kernel="infer_kernel", achieved=r["predict_tflops"],
                         peak=peak, unit="TFLOP/s", frac=r["predict_tflops"] / peak,
                         traffic=None,
                         flop_per_row_member=S.FLOP_PER_ROW_MEMBER,
                         peak_basis="measured bf16 burst" if "bf16_tflops" in peaks
                         else "fallback 1.9 PFLOP/s")
    r["train"] = dict(rows=info["rows"], photons_per_row=info["photons_per_row"],
                      data_seconds=t1 - t0, train_seconds=t2 - t1, members=4,
                      steps_per_member=cfg["steps"], batch=8192,
                      final_loss=[h[-1][1] for h in hist.values()])
    r["mode"] = mode
    return r


def run_table1(mode: str):
    """The network with the paper's inputs (Table 1): random slabs given by optical
    properties (n 1-7, mu_s, mu_a log-uniform, g 0-0.99, d 5-500 um, scattering optical
    depth <= 100), Monte Carlo labels, a 4-member ensemble, held-out slabs against Monte
    Carlo at 1e5 photons."""
    from paper_2409_00165_gb300 import surrogate as S
    cfg = dict(full=dict(train_rows=1000000, train_photons=20000, steps=8000, test_rows=30000),
               quick=dict(train_rows=200000, train_photons=10000, steps=2000,
                          test_rows=10000))[mode]
    r = S.table1_experiment(cfg["train_rows"], cfg["train_photons"], cfg["steps"],
                            cfg["test_rows"], 100000, members=4, seed=40)
    r["mode"] = mode
    return r


def run_stacks():
    """The uneven batch of 64 multilayer stacks x 200 wavelengths (log-uniform 1e4-1e6
    photons each) in one graph-captured launch with an autotuned shape: photon-steps/s."""
    import torch

    from paper_2409_00165_gb300 import fos
    from paper_2409_00165_gb300 import workloads as W
    m = W.layer_stacks()
    dev = "cuda"
    f64 = torch.float64
    d = {k: torch.as_tensor(v, dtype=f64, device=dev) for k, v in W.media_arrays(m).items()}
    wl = torch.as_tensor(m["wl"], dtype=f64, device=dev)
    sg = torch.as_tensor(m["species_group"], dtype=torch.int32, device=dev)
    rad = torch.as_tensor(m["radius"], dtype=f64, device=dev)
    vf = torch.as_tensor(m["vol_frac"], dtype=f64, device=dev)
    n = m["n_groups"] * m["n_wl"]
    mu_s, mu_a, g = (torch.zeros(n, dtype=f64, device=dev) for _ in range(3))
    fos.check(fos.fos_mie_properties(wl, d["nm_re"], d["nm_im"], sg, d["np_re"], d["np_im"],
                                     rad, vf, mu_s, mu_a, g), "mie")
    th = torch.as_tensor(m["thickness"], dtype=f64, device=dev)
    nl = torch.as_tensor(m["n_layers"], dtype=torch.int32, device=dev)
    nph = torch.as_tensor(m["n_photons"], dtype=torch.int64, device=dev)
    sub = torch.as_tensor(m["substrate_R"], dtype=f64, device=dev)
    b = fos.make_batch(m["n_stacks"], m["n_wl"], m["max_layers"], mu_s, mu_a, g, d["nm_re"], th,
                       n_layers=nl, substrate_R=sub, n_photons=nph, seed=m["seed"])
    counts = torch.zeros((m["n_stacks"] * m["n_wl"], fos.FOS_NCOUNT), dtype=torch.int64,
                         device=dev)
    fos.check(fos.fos_mc_spectrum(b, counts, None, 0, fos.FOS_AUTOTUNE), "stacks autotune")
    tun = fos.fos_mc_get_tuning(b)
    a, e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record()
    fos.check(fos.fos_mc_spectrum(b, counts, None, 0, 0), "stacks")
    e.record()
    torch.cuda.synchronize()
    s = a.elapsed_time(e) / 1e3
    c = counts.sum(dim=0).cpu().numpy()
    return dict(items=int(counts.shape[0]), photons=int(c[:4].sum()), photon_steps=int(c[4]),
                seconds=s, photon_steps_per_s=float(c[4]) / s,
                spectra_per_s=m["n_stacks"] / s, tuning=dict(block=tun[0], ppt=tun[1]))


def _mie_mc_leg(m, photons: int, seed: int):
    """Mie (core-shell where the media hold core radii) + effective medium, then the walk
    at `photons` per wavelength, for single-layer stacks in the media dict m; each part
    timed once with CUDA events after a warm-up call."""
    import numpy as np
    import torch

    from paper_2409_00165_gb300 import fos
    from paper_2409_00165_gb300 import workloads as W
    dev = "cuda"
    f64 = torch.float64
    d = {k: torch.as_tensor(v, dtype=f64, device=dev) for k, v in W.media_arrays(m).items()}
    t = lambda a, dt=f64: torch.as_tensor(a, dtype=dt, device=dev)
    wl, sg, rad, vf = t(m["wl"]), t(m["species_group"], torch.int32), t(m["radius"]), t(m["vol_frac"])
    n = m["n_groups"] * m["n_wl"]
    mu_s, mu_a, g = (torch.zeros(n, dtype=f64, device=dev) for _ in range(3))
    if "core_radius" in m:
        nc = np.asarray(m["n_core"])
        cr, nc_re, nc_im = t(m["core_radius"]), t(nc.real.reshape(-1)), t(nc.imag.reshape(-1))
        mie = lambda fl: fos.fos_mie_properties_cs(wl, d["nm_re"], d["nm_im"], sg, d["np_re"],
                                                   d["np_im"], nc_re, nc_im, rad, cr, vf, mu_s,
                                                   mu_a, g, flags=fl)
    else:
        mie = lambda fl: fos.fos_mie_properties(wl, d["nm_re"], d["nm_im"], sg, d["np_re"],
                                                d["np_im"], rad, vf, mu_s, mu_a, g, flags=fl)
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
    fos.check(mie(0), "mie warm-up")
    extra = {k: t(m[k]) for k in ("cos_incidence", "n_below", "k_below") if k in m}
    b = fos.make_batch(m["n_stacks"], m["n_wl"], 1, mu_s, mu_a, g, d["nm_re"], t(m["thickness"]),
                       photons_per_item=photons, seed=seed, **extra)
    counts = torch.zeros((n, fos.FOS_NCOUNT), dtype=torch.int64, device=dev)
    solar = torch.zeros((m["n_stacks"], 3), dtype=f64, device=dev)
    G = t(W.solar_like_irradiance(m["wl"]))
    fos.check(fos.fos_mc_spectrum(b, counts, None, 0, fos.FOS_AUTOTUNE), "mc warm-up")
    torch.cuda.synchronize()
    ev[0].record()
    fos.check(mie(fos.FOS_ASYNC), "mie")
    ev[1].record()
    fos.check(fos.fos_mc_spectrum(b, counts, None, 0, fos.FOS_ASYNC), "mc")
    ev[2].record()
    fos.check(fos.fos_solar_weighted(m["n_stacks"], wl, G, counts, solar, fos.FOS_ASYNC),
              "solar")
    torch.cuda.synchronize()
    fos.check(fos.fos_sync_status(), "mie + mc + solar")
    t_mie, t_mc = ev[0].elapsed_time(ev[1]) / 1e3, ev[1].elapsed_time(ev[2]) / 1e3
    c = counts.sum(dim=0).cpu().numpy()
    evals = len(m["radius"]) * m["n_wl"]
    cn = counts.cpu().numpy().reshape(m["n_stacks"], m["n_wl"], -1)
    refl = (cn[:, :, 0] + cn[:, :, 1]) / photons
    return dict(sizes=len(m["radius"]), mie_evals=evals, mie_seconds=t_mie,
                mie_evals_per_s=evals / t_mie, mc_seconds=t_mc, photons=int(c[:4].sum()),
                photon_steps=int(c[4]), photon_steps_per_s=float(c[4]) / t_mc,
                spectra_per_s=m["n_stacks"] / (t_mie + t_mc),
                mean_reflectance=[float(x) for x in refl.mean(axis=1)],
                solar_weighted_RAT=[[round(float(v), 6) for v in row]
                                    for row in solar.cpu().numpy()])


def run_distributions():
    """Particle-size distributions (each diameter -> 101 Gaussian sizes over D +- 3 sigma):
    silicon-like spheres D = 0.5 um at 0.1 % in 500 um of a water-like matrix, sigma = 0,
    0.05, 0.15 um, 400 wavelengths, 1e6 photons per wavelength; Mie over all 203 sizes,
    the effective medium per distribution, then the walk."""
    from paper_2409_00165_gb300 import fos
    from paper_2409_00165_gb300 import workloads as W
    dists = [fos.fos_size_distribution(0.5, s, 0.001) for s in (0.0, 0.05, 0.15)]
    r = _mie_mc_leg(W.size_distribution_media(dists), 1000000, 9)
    r["sigmas_um"] = [0.0, 0.05, 0.15]
    return r


def run_core_shell():
    """Core-shell spheres: hollow silica-like spheres (air core D = 0.5 um, outer D = 0.7,
    0.9, 1.1 um) and solid ones of the same outer sizes, f = 0.6 in a 50 um layer in air,
    400 wavelengths, 1e6 photons per wavelength."""
    from paper_2409_00165_gb300 import workloads as W
    r = _mie_mc_leg(W.hollow_silica_media(), 1000000, 11)
    r["outer_diameters_um"] = [0.7, 0.9, 1.1]
    r["stacks"] = "3 hollow then 3 solid"
    return r


def run_boundaries():
    """Oblique incidence on a conductor: the paint-layer medium, 50 um thick, on an
    aluminium-like Drude metal, lit at 0, 30 and 60 degrees, 400 wavelengths, 1e6
    photons per wavelength; Eq. 21 totals under a 5778 K blackbody spectrum."""
    from paper_2409_00165_gb300 import workloads as W
    r = _mie_mc_leg(W.oblique_conductor_media(), 1000000, 13)
    r["incidence_deg"] = [0, 30, 60]
    return r


# ------------------------------------------------------------------------ reference arm
def run_reference(args):
    """The oracle, as it stands, timed on the host cores on bounded samples."""
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    from paper_2409_00165_gb300 import workloads as W
    import numpy as np
    m = W.paint_layer(photons=args.photons)
    props = _oracle_props(m)
    cores = os.cpu_count() or 1
    wl_idx = np.linspace(0, m["n_wl"] - 1, 8).round().astype(int)
    budget = min(15.0, 150.0 / max(1, args.steps + args.warmup))
    c0, p0, t0 = oracle_sample(m, props, 64 * cores, cores, wl_idx)
    n = int(max(64 * cores, budget / max(t0 / max(p0, 1), 1e-9) / len(wl_idx)))
    for _ in range(args.warmup):
        oracle_sample(m, props, max(64 * cores, n // 8), cores, wl_idx)
    coll = 0
    secs = 0.0
    for _ in range(args.steps):
        c, p, dt = oracle_sample(m, props, n, cores, wl_idx)
        coll += c
        secs += dt
    value = coll / secs
    sample = (f"8 of 400 wavelengths x {n} photons per step, FP32-mirror oracle walk, "
              f"{cores} host threads")
    line = dict(metric=METRIC, value=value, unit=UNIT, n_gpus=world, steps=args.steps,
                warmup=args.warmup, ms_per_step=secs / args.steps * 1e3, higher_is_better=True,
                scaling="weak", vs_baseline=None, dtype="f32", data="synthetic",
                config=dict(workload=WORKLOAD, sample=sample), impl="reference",
                cpu_baseline=dict(value=value, unit=UNIT, cores=cores, kind="oracle",
                                  sample=sample),
                e2e=dict(value=value, unit=UNIT, h2d_bytes_per_step=0, d2h_bytes_per_step=0))
    print(json.dumps(line), flush=True)


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
    else:
        run_fos(args)


if __name__ == "__main__":
    main()
