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


def fractions(counts, stream=None):
    out = torch.zeros((counts.shape[0], 3), dtype=torch.float32, device=counts.device)
    fos.check(fos.fos_counts_to_fractions(counts, out, stream), "fos_counts_to_fractions")
    return out


class Surrogate:
    """An ensemble of MLP members stored in one device buffer."""

    def __init__(self, n_members: int, feat_stats_device, seed: int = 0, device="cuda"):
        self.n_members = n_members
        self.mb = fos.fos_surrogate_model_bytes()
        self.model = torch.zeros(n_members * self.mb, dtype=torch.uint8, device=device)
        stats = feat_stats_device.cpu().numpy().tolist()
        fos.check(fos.fos_surrogate_init(self.model, n_members, seed, stats), "init")
        self.seed = seed
        self.steps_done = [0] * n_members

    @staticmethod
    def stats_of(features):
        st = torch.zeros(64, dtype=torch.float32, device=features.device)
        fos.check(fos.fos_surrogate_feature_stats(features, st), "feature_stats")
        return st

    def fit(self, features, targets, steps: int, batch: int = 8192, lr: float = 1e-3,
            lr_min: float = 2e-5, members=None, log_every: int = 0):
        """Adam with a cosine learning-rate schedule; returns the loss history."""
        members = range(self.n_members) if members is None else members
        loss = torch.zeros(1, dtype=torch.float32, device=features.device)
        hist = {}
        for k in members:
            hist[k] = []
            for t in range(steps):
                cur = lr_min + 0.5 * (lr - lr_min) * (1 + math.cos(math.pi * t / steps))
                fos.check(fos.fos_surrogate_train_step(
                    self.model, k, features, targets, batch, self.seed, self.steps_done[k], cur,
                    loss_out=loss, flags=fos.FOS_ASYNC), "train_step")
                self.steps_done[k] += 1
                if log_every and (t % log_every == 0 or t == steps - 1):
                    hist[k].append((t, loss.item()))
        fos.check(fos.fos_sync_status(), "training")
        return hist

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
