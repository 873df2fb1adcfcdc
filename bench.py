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
no collective on the data path); with --scaling strong the ranks split the photons of
one spectrum by photon-id ranges and sum their int64 counts with one all-reduce (NCCL)
per step, which gives the single-rank counts bit for bit.  Rank 0 prints one JSON line.
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

# Algorithmic work of one collision event (photon-step): a hand tally of the operations
# the method performs (free path, absorb-or-scatter, Henyey-Greenstein, direction, the
# Philox block of its random numbers), each IEEE +,-,*,fma, compare, select, min/max,
# integer multiply-high or -low, logic op or SFU op counted once, whatever series or
# instruction sequence an implementation uses for log, cos, reciprocal or square root:
#   Philox4x32-10, key schedule hoisted (the key is the seed): 10 rounds x (2 mul.hi +
#     2 mul.lo + 2 three-input xor) + the event counter                              61
#   3 uniforms from words (shift, or, subtract) + the absorption test on a word       10
#   free path -ln u = log2(u) * -ln 2                                                  2
#   collision test tau |mu| < mu_t dist (distance select, 2 products, compares) and
#     the move s = tau / mu_t (reciprocal product), z += mu s                           9
#   Henyey-Greenstein: 2g, 2g u + (1 - g), (1 - g^2) / den (reciprocal + product),
#     1 + g^2 - t^2, / 2g, isotropic test and select, clamp                            10
#   direction: near-vertical test, 1 - mu^2, 1 - cos^2, product, square root (SFU +
#     product), cos(2 pi u) (offset, scale, SFU), mu cos + q cos phi, clamp            13
#   event and collision counters, event cap test, loop                                  4
# I_STEP = 109 issue slots per step, X_STEP = 4 of them on the SFU (log2, reciprocal,
# square root, cosine).  Ceiling (per SM per clock: 4 warp instructions = 128 lanes
# issued, 16 SFU lanes) = SMs x f x min(128 / I_STEP, 16 / X_STEP) photon-steps/s.
I_STEP = 61 + 10 + 2 + 9 + 10 + 13 + 4   # = 109
X_STEP = 4
# The exact walk's own instruction budget is larger: it evaluates -ln u and cos 2 pi u
# by 22- and ~20-operation series (bit-exact with the oracle) and IEEE division/sqrt.
IMPL_OPS_PER_STEP_EXACT = 162


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
    ap.add_argument("--surrogate", choices=["full", "quick", "paper", "off"], default="full",
                    help="surrogate leg (1 GPU only): MC training data, ensemble training, "
                         "design sweep with MC fallback and audit; 'paper' trains on 2e6 "
                         "rows at 1e5 photons each (several GPU-minutes)")
    ap.add_argument("--stacks", choices=["on", "off"], default="on",
                    help="time the uneven multilayer-stack batch (graph-captured, "
                         "autotuned) with both walks")
    ap.add_argument("--scaling", choices=["weak", "strong"], default="weak",
                    help="under torchrun: a spectrum per rank (weak), or one spectrum split "
                         "across the ranks by photon ranges (strong)")
    ap.add_argument("--fast-steps", type=int, default=5,
                    help="steps of the paint layer timed again with the fast (SFU) walk")
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
    # the same oracle on one core, on a smaller sample of the same 8 wavelengths
    per_photon_1 = dt / max(phot, 1) * cores      # one core, from the threaded run
    n1 = int(max(64, min(n, seconds / 3.0 / max(per_photon_1, 1e-9) / 8)))
    c1, p1, t1 = oracle_sample(m, props, n1, 1, wl_idx)
    return dict(value=coll / dt, unit=UNIT, cores=cores, kind="oracle",
                sample=f"8 of 400 wavelengths (evenly spaced) x {n} photons each, FP32-mirror "
                       f"oracle walk, {cores} host threads sharing photon ranges; "
                       f"{coll} photon-steps in {dt:.1f} s",
                photons_per_s=phot / dt,
                single_core=dict(value=c1 / t1, unit=UNIT, cores=1,
                                 sample=f"the same 8 wavelengths x {n1} photons on one thread; "
                                        f"{c1} photon-steps in {t1:.1f} s"))


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

    strong = args.scaling == "strong" and world > 1
    if strong:
        # this rank's photon-id range of every wavelength of the one spectrum
        from paper_2409_00165_gb300 import shard
        pf, pn = shard.photon_ranges(np.full(n_wl, m["photons_per_item"], np.int64), rank, world)
        pf, pn = torch.as_tensor(pf, device=dev), torch.as_tensor(pn, device=dev)

    def step(seed, flags=fos.FOS_ASYNC, ev=None, src=d, mc_flags=0, whole=False):
        fos.check(fos.fos_mie_properties(src["wl"], src["nm_re"], src["nm_im"], src["sg"],
                                         src["np_re"], src["np_im"], src["radius"],
                                         src["vol_frac"], mu_s, mu_a, g,
                                         flags=flags & fos.FOS_ASYNC),
                  "fos_mie_properties")
        split = strong and not whole
        b = fos.make_batch(1, n_wl, 1, mu_s, mu_a, g, src["nm_re"], src["thickness"],
                           photons_per_item=m["photons_per_item"], seed=seed,
                           item_id_base=0 if strong else rank * n_wl,
                           photon_first=pf if split else None, n_photons=pn if split else None)
        if ev is not None:
            ev[0].record(stream)
        fos.check(fos.fos_mc_spectrum(b, counts, None, 0, flags | mc_flags), "fos_mc_spectrum")
        if ev is not None:
            ev[1].record(stream)
        if split:
            shard.allreduce_counts(counts)   # exact int64 sum over the ranks (NCCL)
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
    if strong:   # every rank holds the summed counts of the one spectrum
        coll_all, phot_all = float(coll), float(photons)
    secs = ms_total / 1e3
    value = coll_all / secs
    spectra_per_s = (1 if strong else world) * K / secs
    strong_check = None
    if strong:
        # the last step's summed counts against one rank running the whole spectrum
        if rank == 0:
            last = per_step_counts[K - 1].clone()
            step(2000 + K - 1, flags=0, whole=True)
            strong_check = bool(torch.equal(last, counts))
            assert strong_check, "sharded counts differ from the single-rank run"
        dist.barrier()

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
    sm_count = torch.cuda.get_device_properties(dev).multi_processor_count
    roof = walk_roofline(steps_per_launch / walk_s, sm_count, clocks)
    roof.update(kernel="walk_kernel (exact)", photon_steps_per_launch=steps_per_launch,
                launch_ms=walk_s * 1e3, impl_ops_per_step=IMPL_OPS_PER_STEP_EXACT,
                impl_ops_frac=IMPL_OPS_PER_STEP_EXACT * steps_per_launch / walk_s
                / (sm_count * 128 * roof["f_hz"]))

    # The paint layer's walk load balance: one more exact launch with per-block times.
    tail = None
    try:
        step(5000, flags=0, mc_flags=fos.FOS_RECORD_TIMES)
        tail = tail_stats(fos.fos_mc_walk_times())
    except Exception as exc:
        tail = dict(error=str(exc))

    # The fast (SFU) walk on the same workload: tuned for it, then timed the same way.
    fast = None
    if args.fast_steps > 0 and world == 1:
        try:
            fast = run_fast_walk(args, step, counts, stream, l2, sm_count, clocks, tail_stats)
        except Exception as exc:
            fast = dict(error=str(exc))

    surr = None
    if args.surrogate != "off" and world == 1:
        try:
            surr = run_surrogate(args.surrogate)
        except Exception as exc:  # the surrogate leg must not hide the MC number
            surr = dict(error=str(exc))
    t1 = None
    if args.surrogate != "off" and world == 1:
        try:
            t1 = run_table1("quick" if args.surrogate == "quick" else "full")
        except Exception as exc:
            t1 = dict(error=str(exc))
    stacks = None
    if args.stacks == "on" and world == 1:
        try:
            stacks = run_stacks(sm_count, clocks)
        except Exception as exc:
            stacks = dict(error=str(exc))
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
    # details that would swamp the JSON line go to stderr
    for name, leg in (("surrogate", surr), ("table1_network", t1)):
        if isinstance(leg, dict):
            worst = leg.pop("worst", None) or (leg.get("audit") or {}).pop("worst", None)
            if worst:
                sys.stderr.write(f"{name} worst rows: {json.dumps(worst)}\n")
    line = dict(
        metric=METRIC, value=value, unit=UNIT, n_gpus=world, steps=K, warmup=args.warmup,
        ms_per_step=ms_total / K, higher_is_better=True,
        scaling="strong" if strong else "weak", vs_baseline=None,
        dtype="f32", data="synthetic",
        config=dict(workload=WORKLOAD, photons_per_step=n_wl * m["photons_per_item"],
                    wavelengths=n_wl, l2="flushed before every step by a 512 MiB write "
                    "inside the timed region", tuning=dict(block=tuning[0], ppt=tuning[1]),
                    precision="Mie f64, walk f32 (exact walk), tallies int64",
                    parallelism=(f"photon ranges x{world}, int64 all-reduce" if strong
                                 else f"replicas x{world}")),
        strong_scaling_bit_identical=strong_check,
        spectra_per_s=spectra_per_s, photons_per_s=phot_all / secs,
        photon_steps_per_photon=coll / max(photons, 1),
        e2e=e2e, roofline=roof, cpu_baseline=cpu, clocks=clocks,
        gpu_launches=6 * K,
        gpu_launches_detail="per step: mie_kernel, emt_kernel, pack_kernel, unit_scan_kernel, "
                            "walk_kernel, solar_kernel",
        solar_weighted=dict(zip(("R_s", "A_s", "T_s"), solar.cpu().tolist())),
        walk_tail=tail, size_distributions=dists, core_shell=cs, oblique_conductor=bnd,
        surrogate=surr, table1_network=t1, layer_stacks=stacks, fast_walk=fast,
    )
    line["summary"] = summarize(line)
    print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


def walk_roofline(steps_per_s: float, sm_count: int, clocks):
    """The FP32/INT + SFU issue roofline of the walk at the maximum SM clock."""
    peaks = {}
    try:
        peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        pass
    f_max = float(peaks.get("sm_max_mhz", 2070.0)) * 1e6
    per_clock = min(128.0 / I_STEP, 16.0 / X_STEP)
    ceiling = sm_count * f_max * per_clock
    roof = dict(bound="alu", achieved=steps_per_s, peak=ceiling, unit="photon-steps/s",
                frac=steps_per_s / ceiling, traffic=None, i_step=I_STEP, x_step=X_STEP,
                peak_basis=f"{sm_count} SMs x {f_max / 1e6:.0f} MHz (maximum SM clock) x "
                           f"min(128/{I_STEP}, 16/{X_STEP}) steps per SM per clock",
                f_hz=f_max)
    if clocks and clocks.get("sm_mhz"):
        roof["frac_at_sampled_clock"] = steps_per_s / (sm_count * clocks["sm_mhz"] * 1e6
                                                       * per_clock)
    return roof


def tail_stats(t):
    """Load balance of a persistent walk launch from per-block (start, end) times: the
    launch span, and the tail = the time after half of the blocks have finished."""
    import numpy as np
    if len(t) == 0:
        return None
    t0, t1 = int(t[:, 0].min()), int(t[:, 1].max())
    ends = np.sort(t[:, 1])
    half = int(ends[len(ends) // 2])
    span = max(t1 - t0, 1)
    return dict(blocks=int(len(t)), launch_ms=span / 1e6, tail_ms=(t1 - half) / 1e6,
                tail_frac=(t1 - half) / span,
                first_block_end_frac=(int(ends[0]) - t0) / span)


def run_fast_walk(args, step, counts, stream, l2, sm_count, clocks, tail_fn):
    """The paint layer with the fast (SFU) walk: autotuned, then `fast_steps` steps timed
    (walk launch on the launching stream, L2 flushed before each), then one launch with
    per-block times."""
    import torch
    from paper_2409_00165_gb300 import fos
    step(1500, flags=0 if args.no_autotune else fos.FOS_AUTOTUNE, mc_flags=fos.FOS_FAST_WALK)
    step(1501, mc_flags=fos.FOS_FAST_WALK)
    torch.cuda.synchronize()
    K = args.fast_steps
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
           for _ in range(K)]
    coll = 0
    for k in range(K):
        l2.fill_(float(k))
        step(6000 + k, ev=evs[k], mc_flags=fos.FOS_FAST_WALK)
        torch.cuda.synchronize()
        coll += int(counts[:, 4].sum())
    fos.check(fos.fos_sync_status(stream), "fast walk")
    walk_s = sum(a.elapsed_time(b) for a, b in evs) / 1e3
    b = step(1502, flags=0, mc_flags=fos.FOS_FAST_WALK)
    tun = fos.fos_mc_get_tuning(b, fos.FOS_FAST_WALK)
    step(1503, flags=0, mc_flags=fos.FOS_FAST_WALK | fos.FOS_RECORD_TIMES)
    roof = walk_roofline(coll / walk_s, sm_count, clocks)
    return dict(photon_steps_per_s=coll / walk_s, steps=K, launch_ms=walk_s / K * 1e3,
                roofline=dict(frac=roof["frac"], peak=roof["peak"],
                              frac_at_sampled_clock=roof.get("frac_at_sampled_clock")),
                tuning=dict(block=tun[0], ppt=tun[1]), tail=tail_fn(fos.fos_mc_walk_times()))


def summarize(line: dict) -> dict:
    """The headline numbers of every leg in one short dict (printed last on the line)."""
    def get(d, *ks):
        for k in ks:
            if not isinstance(d, dict):
                return None
            d = d.get(k)
        return d

    def r(v, n=4):
        return None if v is None else float(f"{v:.{n}g}")

    surr, t1, st, fw = (line.get("surrogate"), line.get("table1_network"),
                        line.get("layer_stacks"), line.get("fast_walk"))
    return dict(
        walk_exact=dict(photon_steps_per_s=r(line["value"]),
                        frac=r(get(line, "roofline", "frac"), 3),
                        tail_frac=r(get(line, "walk_tail", "tail_frac"), 3)),
        walk_fast=None if not isinstance(fw, dict) or "error" in fw else dict(
            photon_steps_per_s=r(fw["photon_steps_per_s"]), frac=r(fw["roofline"]["frac"], 3),
            speedup_vs_exact_launch=r(line["roofline"]["launch_ms"] / fw["launch_ms"], 3)),
        layer_stacks=None if not isinstance(st, dict) or "error" in st else dict(
            photon_steps_per_s=r(get(st, "exact", "photon_steps_per_s")),
            spectra_per_s=r(get(st, "exact", "spectra_per_s")),
            tuned=get(st, "exact", "tuning"), tuned_vs_fixed_128x8=r(st.get("tuned_speedup"), 3),
            tail_frac=r(get(st, "exact", "tail", "tail_frac"), 3),
            fast_photon_steps_per_s=r(get(st, "fast", "photon_steps_per_s"))),
        surrogate=None if not isinstance(surr, dict) or "error" in surr else dict(
            mode=surr.get("mode"), train_rows=get(surr, "train", "rows"),
            train_photons=get(surr, "train", "photons_per_row"),
            spectra_per_s=r(surr.get("spectra_per_s")),
            mc_spectra_per_s=r(surr.get("mc_spectra_per_s")),
            speedup_vs_mc=r(surr.get("speedup_vs_mc")),
            audit_rows=get(surr, "audit", "rows"),
            audit_max=[r(v, 3) for v in get(surr, "audit", "max") or []],
            audit_mae=[r(v, 3) for v in get(surr, "audit", "mae") or []],
            audit_refined_max=[r(v, 3) for v in get(surr, "audit", "refined", "max") or []],
            flagged_rows=surr.get("flagged"),
            infer_frac=r(get(surr, "roofline", "frac"), 3)),
        table1_network=None if not isinstance(t1, dict) or "error" in t1 else dict(
            max=[r(v, 3) for v in t1.get("max") or []],
            mae=[r(v, 3) for v in t1.get("mae") or []]),
    )


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
               # the surrogate-training workload at its stated size: 2e6 (design, wavelength)
               # rows at 1e5 photons each
               paper=dict(designs=40000, blocks=20, wl=50, photons=100000, steps=30000,
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
                audit_frac=0.001 if mode == "quick" else 0.01)
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
                      data_seconds=t1 - t0, data_mc_seconds=info["mc_seconds"],
                      data_photon_steps_per_s=info["photon_steps"] / max(info["mc_seconds"], 1e-9),
                      train_seconds=t2 - t1, members=4,
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


def run_stacks(sm_count: int, clocks):
    """The uneven batch of 64 multilayer stacks x 200 wavelengths (1-3 layers on a 5 %
    reflector, log-uniform 1e4-1e6 photons per item), one graph-captured persistent walk
    launch per call: exact and fast walk, each autotuned (block x photons per thread on a
    proportionally scaled copy of the batch) and timed over 3 launches with CUDA events;
    the exact walk also at the fixed default shape (128 threads, 8 photons per thread);
    per-block times give the launch's tail."""
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

    def timed(flags, reps=3):
        fos.check(fos.fos_mc_spectrum(b, counts, None, 0, flags), "stacks warm-up")
        ms = []
        for _ in range(reps):
            a, e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record()
            fos.check(fos.fos_mc_spectrum(b, counts, None, 0, flags | fos.FOS_ASYNC), "stacks")
            e.record()
            torch.cuda.synchronize()
            ms.append(a.elapsed_time(e))
        fos.check(fos.fos_sync_status(), "stacks")
        c = counts.sum(dim=0).cpu().numpy()
        sec = statistics.mean(ms) / 1e3
        return dict(seconds=sec, photon_steps=int(c[4]), photons=int(c[:4].sum()),
                    photon_steps_per_s=float(c[4]) / sec, spectra_per_s=m["n_stacks"] / sec)

    out = dict(items=int(counts.shape[0]))
    fos.fos_mc_set_tuning(128, 8)
    fixed = timed(0)
    fos.fos_mc_set_tuning(0, 0)
    for name, fl in (("exact", 0), ("fast", fos.FOS_FAST_WALK)):
        t0 = time.perf_counter()
        fos.check(fos.fos_mc_spectrum(b, counts, None, 0, fos.FOS_AUTOTUNE | fl), "autotune")
        tune_s = time.perf_counter() - t0
        r = timed(fl)
        tun = fos.fos_mc_get_tuning(b, fl)
        r["tuning"] = dict(block=tun[0], ppt=tun[1])
        r["autotune_seconds"] = tune_s
        fos.check(fos.fos_mc_spectrum(b, counts, None, 0, fl | fos.FOS_RECORD_TIMES), "times")
        r["tail"] = tail_stats(fos.fos_mc_walk_times())
        r["roofline_frac"] = walk_roofline(r["photon_steps_per_s"], sm_count, clocks)["frac"]
        out[name] = r
    out["fixed_128x8"] = dict(seconds=fixed["seconds"],
                              photon_steps_per_s=fixed["photon_steps_per_s"])
    out["tuned_speedup"] = fixed["seconds"] / out["exact"]["seconds"]
    out["photons"] = out["exact"]["photons"]
    return out


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
