"""Surrogate workflow on the C ABI: Monte Carlo training data, ensemble training,
surrogate design sweep with Monte Carlo fallback (arxiv 2409.00165, section "Photon
transport": a network trained on Monte Carlo simulations replaces the walk, within the
ranges it was trained on, Table 1).

Each function only moves arguments between calls of libfos; every step of the method
(Mie, effective medium, photon walk, features, training, inference) runs in the library.
"""
from __future__ import annotations

import math

import numpy as np
import torch

from . import fos
from . import workloads as W

F64 = torch.float64
# Algorithmic multiply-adds x 2 of one row through one member (real layer shapes
# 9-256-256-256-256-3, padding excluded).
FLOP_PER_ROW_MEMBER = 2 * (9 * 256 + 3 * 256 * 256 + 256 * 3)


class Media:
    """Single-layer designs (one particle species per design) on a wavelength grid, as
    device tensors in the layouts of fos_mie_properties / fos_mc_spectrum."""

    def __init__(self, radius, vol_frac, thickness, wl, device="cuda"):
        radius = np.asarray(radius, np.float64)
        n_d, n_wl = radius.size, len(wl)
        self.n_designs, self.n_wl = n_d, n_wl
        dev = torch.device(device)
        nm = W.matrix_index(wl)
        npi = W.particle_index(wl)
        t = lambda a: torch.as_tensor(np.ascontiguousarray(a), dtype=F64, device=dev)
        self.wl = t(wl)
        self.nm_re = t(np.broadcast_to(nm.real, (n_d, n_wl)).reshape(-1))
        self.nm_im = t(np.broadcast_to(nm.imag, (n_d, n_wl)).reshape(-1))
        self.np_re = t(np.broadcast_to(npi.real, (n_d, n_wl)).reshape(-1))
        self.np_im = t(np.broadcast_to(npi.imag, (n_d, n_wl)).reshape(-1))
        self.species_group = torch.arange(n_d, dtype=torch.int32, device=dev)
        self.radius = t(radius)
        self.vol_frac = t(vol_frac)
        self.thickness = t(thickness)
        self.mu_s = torch.zeros(n_d * n_wl, dtype=F64, device=dev)
        self.mu_a = torch.zeros_like(self.mu_s)
        self.g = torch.zeros_like(self.mu_s)

    @property
    def rows(self) -> int:
        return self.n_designs * self.n_wl

    def mie(self, flags=0, stream=None):
        fos.check(fos.fos_mie_properties(self.wl, self.nm_re, self.nm_im, self.species_group,
                                         self.np_re, self.np_im, self.radius, self.vol_frac,
                                         self.mu_s, self.mu_a, self.g, flags=flags, stream=stream),
                  "fos_mie_properties")

    def batch(self, photons: int, seed: int, item_list=None, item_id_base=0):
        return fos.make_batch(self.n_designs, self.n_wl, 1, self.mu_s, self.mu_a, self.g,
                              self.nm_re, self.thickness, photons_per_item=photons, seed=seed,
                              item_list=item_list, item_id_base=item_id_base)

    def mc(self, photons: int, seed: int, item_list=None, flags=0, stream=None):
        b = self.batch(photons, seed, item_list)
        n = item_list.numel() if item_list is not None else self.rows
        counts = torch.zeros((max(n, 1), fos.FOS_NCOUNT), dtype=torch.int64,
                             device=self.mu_s.device)
        fos.check(fos.fos_mc_spectrum(b, counts, None, 0, flags, stream), "fos_mc_spectrum",
                  allow=(fos.FOS_OK,))
        return counts[:n]

    def features(self, flags=0, stream=None):
        out = torch.zeros((self.rows, 9), dtype=torch.float32, device=self.mu_s.device)
        fos.check(fos.fos_surrogate_features(self.wl, self.np_re, self.np_im, self.radius,
                                             self.vol_frac, self.thickness, self.g, self.mu_s,
                                             self.mu_a, out, flags=flags, stream=stream),
                  "fos_surrogate_features")
        return out


def fractions(counts, stream=None, rows=None, out=None):
    if out is None:
        out = torch.zeros((counts.shape[0], 3), dtype=torch.float32, device=counts.device)
    fos.check(fos.fos_counts_to_fractions(counts, out, rows, stream), "fos_counts_to_fractions")
    return out


def flagged_rows(needs):
    rows = torch.empty(needs.numel(), dtype=torch.int32, device=needs.device)
    count = torch.zeros(1, dtype=torch.int64, device=needs.device)
    fos.check(fos.fos_mask_to_rows(needs, rows, count), "fos_mask_to_rows")
    return rows[: int(count.item())]


class Surrogate:
    """An ensemble of MLP members stored in one device buffer."""

    def __init__(self, n_members: int, feat_stats, seed: int = 0, device="cuda"):
        """feat_stats: the 64 statistics floats, a device tensor or a host sequence."""
        self.n_members = n_members
        self.mb = fos.fos_surrogate_model_bytes()
        self.model = torch.zeros(n_members * self.mb, dtype=torch.uint8, device=device)
        if isinstance(feat_stats, torch.Tensor):
            feat_stats = feat_stats.cpu().numpy()
        stats = [float(v) for v in feat_stats]
        fos.check(fos.fos_surrogate_init(self.model, n_members, seed, stats), "init")
        self.seed = seed
        self.steps_done = [0] * n_members

    @staticmethod
    def stats_of(features):
        st = torch.zeros(64, dtype=torch.float32, device=features.device)
        fos.check(fos.fos_surrogate_feature_stats(features, st), "feature_stats")
        return st

    def fit(self, features, targets, steps: int, batch: int = 8192, lr: float = 1e-3,
            lr_min: float = 2e-5, members=None, log_every: int = 0, schedule_steps=None):
        """Adam with a cosine learning-rate schedule over schedule_steps (default: this
        call's steps), taken at each member's global step count, so that a run split into
        several calls, or resumed from a checkpoint, follows the same schedule.  Returns
        the loss history."""
        members = list(range(self.n_members) if members is None else members)
        total = schedule_steps or steps
        dev = features.device
        if members == list(range(self.n_members)) and len(set(self.steps_done)) == 1:
            return self._fit_graph(features, targets, steps, batch, lr, lr_min, log_every,
                                   0 if schedule_steps else self.steps_done[0], total)
        # members in different workspace slots (member mod 4) step concurrently, one
        # stream per slot; a member's own steps stay in order on its slot's stream
        streams = {k % 4: torch.cuda.Stream(device=dev) for k in members}
        loss = {k: torch.zeros(1, dtype=torch.float32, device=dev) for k in members}
        hist = {k: [] for k in members}
        cur_stream = torch.cuda.current_stream(dev)
        for st in streams.values():
            st.wait_stream(cur_stream)
        for t in range(steps):
            for k in members:
                g = min(self.steps_done[k], total) if schedule_steps else t
                cur = lr_min + 0.5 * (lr - lr_min) * (1 + math.cos(math.pi * g / total))
                fos.check(fos.fos_surrogate_train_step(
                    self.model, k, features, targets, batch, self.seed, self.steps_done[k], cur,
                    loss_out=loss[k], flags=fos.FOS_ASYNC, stream=streams[k % 4]),
                    "train_step")
                self.steps_done[k] += 1
                if log_every and (t % log_every == 0 or t == steps - 1):
                    streams[k % 4].synchronize()
                    hist[k].append((t, loss[k].item()))
        for st in streams.values():
            cur_stream.wait_stream(st)
        torch.cuda.synchronize(dev)
        fos.check(fos.fos_sync_status(), "training")
        return hist

    def _fit_graph(self, features, targets, steps, batch, lr, lr_min, log_every, origin, total):
        """All members together, one graph launch per step (fos_surrogate_fit); the loss is
        read back at the logging steps only."""
        dev = features.device
        loss = torch.zeros(self.n_members, dtype=torch.float32, device=dev)
        hist = {k: [] for k in range(self.n_members)}
        marks = sorted({t for t in range(steps) if log_every and (t % log_every == 0
                                                                  or t == steps - 1)})
        done = 0
        for t in marks + [steps - 1]:
            n = t + 1 - done
            if n <= 0:
                continue
            fos.check(fos.fos_surrogate_fit(self.model, self.n_members, features, targets,
                                            batch, self.seed, n, lr, lr_min, origin, total,
                                            loss_out=loss, flags=fos.FOS_ASYNC), "fit")
            done += n
            if t in marks:
                vals = loss.cpu().tolist()
                for k in range(self.n_members):
                    hist[k].append((t, vals[k]))
        torch.cuda.synchronize(dev)
        fos.check(fos.fos_sync_status(), "training")
        self.steps_done = [s + steps for s in self.steps_done]
        return hist

    def save(self, path: str):
        """Checkpoint: the whole model buffer (FP32 parameters, Adam state, BF16 copies,
        weight image, feature statistics) and the step counts, as an .npz file."""
        torch.cuda.synchronize()
        np.savez(path, model=self.model.cpu().numpy(), steps_done=np.array(self.steps_done),
                 seed=self.seed, n_members=self.n_members, model_bytes=self.mb,
                 api=fos.lib().fos_api_version())

    @classmethod
    def restore(cls, path: str, device="cuda"):
        """A surrogate continued from a checkpoint written by save()."""
        z = np.load(path)
        if int(z["model_bytes"]) != fos.fos_surrogate_model_bytes():
            raise ValueError("checkpoint model layout differs from this library's")
        sur = cls.__new__(cls)
        sur.n_members = int(z["n_members"])
        sur.mb = int(z["model_bytes"])
        sur.seed = int(z["seed"])
        sur.steps_done = [int(v) for v in z["steps_done"]]
        sur.model = torch.as_tensor(z["model"]).to(device)
        return sur

    def predict(self, features, threshold: float = 0.01, n_members=None, flags=0, stream=None):
        n = features.shape[0]
        dev = features.device
        rat = torch.zeros((n, 3), dtype=torch.float32, device=dev)
        spread = torch.zeros(n, dtype=torch.float32, device=dev)
        needs = torch.zeros(n, dtype=torch.uint8, device=dev)
        fos.check(fos.fos_surrogate_predict(self.model, n_members or self.n_members, features, rat,
                                            spread, needs, threshold, flags=flags, stream=stream),
                  "fos_surrogate_predict")
        return rat, spread, needs


def training_set(n_designs: int, wl_per_block: int, blocks: int, photons: int, seed: int,
                 device="cuda", log_share: float = 0.0):
    """Monte Carlo training rows of single-layer designs (workload ranges of r, f, d).

    The designs are split into `blocks`; each block gets its own sorted random
    wavelength set drawn from U(0.3, 2.5) um plus both ends of that range, so that the
    training rows cover the whole spectrum.  Returns (features, fractions, info)."""
    rng = np.random.default_rng(seed)
    d = W.single_layer_designs(n_designs, seed=seed, n_wl=None, log_share=log_share)
    per = n_designs // blocks
    feats, targs = [], []
    coll = phot = 0
    mc_s = 0.0
    for k in range(blocks):
        sl = slice(k * per, (k + 1) * per)
        wl = np.sort(np.concatenate([[0.3, 2.5], rng.uniform(0.3, 2.5, wl_per_block - 2)]))
        m = Media(d["radius"][sl], d["vol_frac"][sl], d["thickness"][sl], wl, device)
        m.mie()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        counts = m.mc(photons, seed=seed * 1000 + k)
        b.record()
        torch.cuda.synchronize()
        mc_s += a.elapsed_time(b) / 1e3
        tot = counts.sum(dim=0)
        coll += int(tot[4].item())
        phot += int(tot[:4].sum().item())
        feats.append(m.features())
        targs.append(fractions(counts))
    info = dict(rows=per * blocks * wl_per_block, designs=per * blocks, photons_per_row=photons,
                mc_seconds=mc_s, photon_steps=coll, photons=phot)
    return torch.cat(feats), torch.cat(targs), info


def sweep(sur: Surrogate, n_designs: int, n_wl: int, seed: int, threshold: float = 0.01,
          fallback_photons: int = 100000, audit_frac: float = 0.001, audit_photons: int = 100000,
          refine_rows: int = 64, device="cuda"):
    """Surrogate design sweep: Mie -> features -> ensemble prediction -> Monte Carlo on the
    rows the ensemble flags; then a random audit of rows by Monte Carlo.  Returns timings,
    counts and the audit errors (absolute, per R, A, T) of the final spectra."""
    d = W.single_layer_designs(n_designs, seed=seed, n_wl=n_wl)
    m = Media(d["radius"], d["vol_frac"], d["thickness"], d["wl"], device)
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(5)]
    torch.cuda.synchronize()
    ev[0].record()
    m.mie(flags=fos.FOS_ASYNC)
    f = m.features(flags=fos.FOS_ASYNC)
    ev[1].record()
    rat, spread, needs = sur.predict(f, threshold, flags=fos.FOS_ASYNC)
    ev[2].record()
    flagged = flagged_rows(needs)
    n_flag = int(flagged.numel())
    if n_flag:
        cf = m.mc(fallback_photons, seed=seed + 17, item_list=flagged)
        fractions(cf, rows=flagged, out=rat)
    ev[3].record()
    torch.cuda.synchronize()
    fos.check(fos.fos_sync_status(), "sweep")
    t_mie = ev[0].elapsed_time(ev[1]) / 1e3
    t_pred = ev[1].elapsed_time(ev[2]) / 1e3
    t_fb = ev[2].elapsed_time(ev[3]) / 1e3
    total = t_mie + t_pred + t_fb
    out = dict(designs=n_designs, wavelengths=n_wl, rows=m.rows, flagged=n_flag,
               mie_features_s=t_mie, predict_s=t_pred, fallback_mc_s=t_fb, total_s=total,
               spectra_per_s=n_designs / total,
               spectra_per_s_no_fallback=n_designs / (t_mie + t_pred),
               predict_tflops=FLOP_PER_ROW_MEMBER * m.rows * sur.n_members / t_pred / 1e12)
    if audit_frac > 0:
        arng = np.random.default_rng(seed + 99)
        n_aud = max(1, int(m.rows * audit_frac))
        rows = np.sort(arng.choice(m.rows, size=n_aud, replace=False)).astype(np.int32)
        rt = torch.as_tensor(rows, device=device)
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        ca = m.mc(audit_photons, seed=seed + 23, item_list=rt)
        b.record()
        torch.cuda.synchronize()
        t_a = a.elapsed_time(b) / 1e3
        ya = fractions(ca)
        err = (rat[rt.long()] - ya).abs()
        phot = int(ca[:, :4].sum().item())
        e_all = err.max(dim=1).values
        # binomial standard deviation of the audit's own MC fractions, the floor under any
        # error measured against it
        sig = (ya * (1 - ya) / audit_photons).sqrt().max(dim=1).values
        out["audit"] = dict(rows=n_aud, photons=audit_photons,
                            mae=err.mean(dim=0).cpu().tolist(),
                            max=err.max(dim=0).values.cpu().tolist(),
                            p999=float(torch.quantile(e_all.float(), 0.999).item()),
                            frac_above_0p01=float((e_all > 0.01).float().mean().item()),
                            mc_noise_sigma_max=float(sig.max().item()))
        # the worst audited rows again, against Monte Carlo at 10x the photons (a tenth of
        # the variance): the audit's own noise is part of its largest errors
        k = min(refine_rows, n_aud)
        if k > 0:
            worst = torch.topk(e_all, k).indices
            rows_w = torch.sort(rt[worst]).values.contiguous()
            yw = fractions(m.mc(audit_photons * 10, seed=seed + 29, item_list=rows_w))
            ew = (rat[rows_w.long()] - yw).abs()
            emax = ew.max(dim=1).values
            out["audit"]["refined"] = dict(rows=k, photons=audit_photons * 10,
                                           max=ew.max(dim=0).values.cpu().tolist(),
                                           above_0p01=int((emax > 0.01).sum().item()))
            # the designs of the worst refined rows: where the network is weakest
            top = torch.topk(emax, min(8, k)).indices
            rw = rows_w[top].cpu().numpy()
            dd, ww = rw // n_wl, rw % n_wl
            out["audit"]["worst"] = [
                dict(wl=float(d["wl"][w]), radius=float(d["radius"][i]),
                     vol_frac=float(d["vol_frac"][i]), thickness=float(d["thickness"][i]),
                     err=[round(float(v), 5) for v in ew[j].cpu().tolist()],
                     spread=float(spread[int(r)].item()))
                for i, w, j, r in zip(dd, ww, top.cpu().tolist(), rw)]
        # plain GPU Monte Carlo on the same designs, per spectrum of n_wl wavelengths
        out["mc_photons_per_s"] = phot / t_a
        out["mc_spectra_per_s"] = phot / t_a / (n_wl * audit_photons)
        out["speedup_vs_mc"] = out["spectra_per_s"] / out["mc_spectra_per_s"]
    return out


# ----------------------------------------------------------------------------------
# The network with the paper's own inputs (Table 1): slabs given by optical properties.
# ----------------------------------------------------------------------------------
class Slabs:
    """Homogeneous slabs in air, one row each, as device tensors."""

    def __init__(self, rows: dict, device="cuda"):
        t = lambda a: torch.as_tensor(np.ascontiguousarray(a), dtype=F64, device=device)
        self.n, self.mu_s, self.mu_a = t(rows["n"]), t(rows["mu_s"]), t(rows["mu_a"])
        self.g, self.d = t(rows["g"]), t(rows["d"])
        self.rows = int(self.n.numel())

    def mc(self, photons: int, seed: int, item_list=None, flags=0):
        b = fos.make_batch(self.rows, 1, 1, self.mu_s, self.mu_a, self.g, self.n, self.d,
                           photons_per_item=photons, seed=seed, item_list=item_list)
        n = item_list.numel() if item_list is not None else self.rows
        counts = torch.zeros((max(n, 1), fos.FOS_NCOUNT), dtype=torch.int64,
                             device=self.n.device)
        fos.check(fos.fos_mc_spectrum(b, counts, None, 0, flags), "fos_mc_spectrum")
        return counts[:n]

    def features(self, flags=0):
        out = torch.zeros((self.rows, 9), dtype=torch.float32, device=self.n.device)
        fos.check(fos.fos_surrogate_features_slab(self.n, self.mu_s, self.mu_a, self.g, self.d,
                                                  out, flags=flags),
                  "fos_surrogate_features_slab")
        return out


def table1_stats(features) -> list:
    """Feature statistics of the training rows with the range gate set to Table 1 (and
    the optical-depth cap): rows outside it are flagged for Monte Carlo."""
    st = Surrogate.stats_of(features).cpu().numpy().astype(np.float64)
    T = W.TABLE1
    # features 5-8 are functions of the first five; their bounds only admit every value
    # the Table 1 box can produce, except the scattering depth, capped at tau_s_max
    lo = [T["n"][0], math.log10(T["mu_s"][0] + 1e-4), math.log10(T["mu_a"][0] + 1e-4),
          T["g"][0], math.log10(T["d"][0]), -6.0, -6.0,
          math.log10(1.0 - T["g"][1] + 1e-3), -6.0]
    hi = [T["n"][1], math.log10(T["mu_s"][1] + 1e-4), math.log10(T["mu_a"][1] + 1e-4),
          T["g"][1], math.log10(T["d"][1]), math.log10(T["tau_s_max"] + 1e-6),
          math.log10(T["mu_a"][1] * T["d"][1] + 1e-6), math.log10(1.0 - T["g"][0] + 1e-3),
          math.log10(T["tau_s_max"] + 1e-6)]
    # float32 rounding of a boundary must not flag the boundary itself
    st[32:41] = np.nextafter(np.float32(lo), np.float32(-np.inf))
    st[48:57] = np.nextafter(np.float32(hi), np.float32(np.inf))
    return st.astype(np.float32).tolist()


def table1_experiment(train_rows: int, train_photons: int, steps: int, test_rows: int,
                      test_photons: int, members: int = 4, seed: int = 40, batch: int = 8192,
                      threshold: float = 0.01, device="cuda"):
    """Trains an ensemble on Monte Carlo fractions of random Table 1 slabs and evaluates it
    on held-out slabs against Monte Carlo at test_photons: accuracy, flagged rows, and
    slab evaluations per second of the network (with fallback) against Monte Carlo."""
    tr = Slabs(W.table1_slabs(train_rows, seed, g_log_share=0.5, n_log_share=0.3), device)
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
    ev[0].record()
    y = fractions(tr.mc(train_photons, seed=seed + 1))
    ev[1].record()
    f = tr.features()
    torch.cuda.synchronize()
    t_data = ev[0].elapsed_time(ev[1]) / 1e3
    sur = Surrogate(members, table1_stats(f), seed=seed, device=device)
    t0 = torch.cuda.Event(enable_timing=True)
    t1 = torch.cuda.Event(enable_timing=True)
    t0.record()
    hist = sur.fit(f, y, steps=steps, batch=batch, lr=2e-3, log_every=max(steps - 1, 1))
    t1.record()
    torch.cuda.synchronize()
    t_train = t0.elapsed_time(t1) / 1e3
    te = Slabs(W.table1_slabs(test_rows, seed + 7), device)
    e = [torch.cuda.Event(enable_timing=True) for _ in range(4)]
    e[0].record()
    ft = te.features(flags=fos.FOS_ASYNC)
    rat, spread, needs = sur.predict(ft, threshold, flags=fos.FOS_ASYNC)
    e[1].record()
    flagged = flagged_rows(needs)
    n_flag = int(flagged.numel())
    if n_flag:
        cf = te.mc(test_photons, seed=seed + 11, item_list=flagged)
        fractions(cf, rows=flagged, out=rat)
    e[2].record()
    yt = fractions(te.mc(test_photons, seed=seed + 13))
    e[3].record()
    torch.cuda.synchronize()
    fos.check(fos.fos_sync_status(), "table1")
    t_pred = e[0].elapsed_time(e[1]) / 1e3
    t_fb = e[1].elapsed_time(e[2]) / 1e3
    t_mc = e[2].elapsed_time(e[3]) / 1e3
    err = (rat - yt).abs()
    emax = err.max(dim=1).values
    top = torch.topk(emax, min(8, test_rows)).indices
    rows_t = torch.sort(top).values.to(torch.int32).contiguous()
    # the worst rows again at 10x the photons, with their inputs
    yr = fractions(te.mc(test_photons * 10, seed=seed + 17, item_list=rows_t))
    er = (rat[rows_t.long()] - yr).abs()
    worst = [dict(n=float(te.n[i]), mu_s=float(te.mu_s[i]), mu_a=float(te.mu_a[i]),
                  g=float(te.g[i]), d=float(te.d[i]),
                  err=[round(float(v), 5) for v in er[j].cpu().tolist()],
                  spread=float(spread[i].item()))
             for j, i in enumerate(rows_t.long().cpu().tolist())]
    return dict(train_rows=train_rows, train_photons=train_photons, data_seconds=t_data,
                members=members, steps=steps, train_seconds=t_train,
                final_loss=[h[-1][1] for h in hist.values()],
                test_rows=test_rows, test_photons=test_photons, flagged=n_flag,
                mae=err.mean(dim=0).cpu().tolist(), max=err.max(dim=0).values.cpu().tolist(),
                nn_rows_per_s=test_rows / (t_pred + t_fb),
                nn_rows_per_s_no_fallback=test_rows / t_pred,
                mc_rows_per_s=test_rows / t_mc, speedup_vs_mc=t_mc / (t_pred + t_fb),
                refined_max=er.max(dim=0).values.cpu().tolist(), worst=worst)


def _predict_demo(rows: int, members: int, reps: int):
    """Ensemble prediction on random in-range features (a profiling target)."""
    rng = np.random.default_rng(0)
    x = np.column_stack([rng.uniform(0.3, 2.5, rows), rng.uniform(2.5, 3.1, rows),
                         rng.uniform(-4, -0.3, rows), rng.uniform(0.05, 1, rows),
                         rng.uniform(0.01, 0.3, rows), rng.uniform(1, 2.7, rows),
                         rng.uniform(0, 0.9, rows), rng.uniform(-1, 3, rows),
                         rng.uniform(-4, 2, rows)]).astype(np.float32)
    f = torch.as_tensor(x, device="cuda").contiguous()
    sur = Surrogate(members, Surrogate.stats_of(f), seed=1)
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    for _ in range(2):
        sur.predict(f)
    a.record()
    for _ in range(reps):
        sur.predict(f)
    b.record()
    torch.cuda.synchronize()
    s = a.elapsed_time(b) / 1e3 / reps
    flops = float(FLOP_PER_ROW_MEMBER) * rows * members
    print(f"predict {rows} rows x {members} members: {s * 1e3:.3f} ms, "
          f"{flops / s / 1e12:.1f} TFLOP/s (algorithmic)")


def _mie_demo(designs: int, n_wl: int, reps: int):
    """Mie + effective medium over single-layer designs (a profiling target)."""
    d = W.single_layer_designs(designs, seed=5, n_wl=n_wl)
    m = Media(d["radius"], d["vol_frac"], d["thickness"], d["wl"])
    for _ in range(2):
        m.mie()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record()
    for _ in range(reps):
        m.mie(flags=fos.FOS_ASYNC)
    b.record()
    torch.cuda.synchronize()
    fos.check(fos.fos_sync_status(), "mie demo")
    s = a.elapsed_time(b) / 1e3 / reps
    print(f"mie {m.rows} evaluations: {s * 1e3:.3f} ms, {m.rows / s:.3e} evaluations/s")


def _train_demo(rows: int, members: int, steps: int, batch: int):
    """Graph-captured ensemble training on synthetic rows (a profiling target): features in
    the sweep's ranges, Dirichlet targets; 5 warm-up steps, then `steps` timed."""
    import time
    rng = np.random.default_rng(1)
    x = np.column_stack([rng.uniform(0.3, 2.5, rows), rng.uniform(2.5, 3.1, rows),
                         rng.uniform(-4, -0.3, rows), rng.uniform(0.05, 1, rows),
                         rng.uniform(0.01, 0.3, rows), rng.uniform(1, 2.7, rows),
                         rng.uniform(0, 0.9, rows), rng.uniform(-1, 3, rows),
                         rng.uniform(-4, 2, rows)])
    y = rng.dirichlet(np.ones(3), size=rows)
    f = torch.as_tensor(x, dtype=torch.float32).cuda().contiguous()
    t = torch.as_tensor(y, dtype=torch.float32).cuda().contiguous()
    sur = Surrogate(members, Surrogate.stats_of(f), seed=3)
    sur.fit(f, t, steps=5, batch=batch, lr=2e-3)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    sur.fit(f, t, steps=steps, batch=batch, lr=2e-3)
    torch.cuda.synchronize()
    dt = time.perf_counter() - t0
    flop = 3.0 * FLOP_PER_ROW_MEMBER * batch * members * steps
    print(f"train {members} members x {steps} steps, batch {batch}: {dt / steps * 1e3:.3f} ms "
          f"per ensemble step, {flop / dt / 1e12:.1f} TFLOP/s")


if __name__ == "__main__":
    import argparse
    ap = argparse.ArgumentParser()
    ap.add_argument("--predict-demo", action="store_true")
    ap.add_argument("--mie-demo", action="store_true")
    ap.add_argument("--train-demo", action="store_true")
    ap.add_argument("--steps", type=int, default=300)
    ap.add_argument("--batch", type=int, default=8192)
    ap.add_argument("--designs", type=int, default=10000)
    ap.add_argument("--wl", type=int, default=300)
    ap.add_argument("--rows", type=int, default=1 << 19)
    ap.add_argument("--members", type=int, default=4)
    ap.add_argument("--reps", type=int, default=3)
    a = ap.parse_args()
    if a.predict_demo:
        _predict_demo(a.rows, a.members, a.reps)
    if a.mie_demo:
        _mie_demo(a.designs, a.wl, a.reps)
    if a.train_demo:
        _train_demo(a.rows, a.members, a.steps, a.batch)
