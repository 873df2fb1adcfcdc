"""The GPU walk at the benchmark's own size and optical depth against the definition.

The photon-for-photon tests compare the GPU walk with the oracle's FP32 mirror, which
shares the kernel's operation order and random layout.  These tests judge it instead
against two references that share neither:

  * the oracle's definition walk (FP64, the order of section "Photon transport", its
    own sequential random stream), run at an independent seed;
  * the discrete-ordinates solution of the transfer equation (`rte_dom.slab_rat`, a
    deterministic method), for the homogeneous paint layer.

on the full 400-wavelength x 1e6-photon paint layer (tau_d up to 525, albedo up to
0.9995, about 230 collisions per photon) in the benchmark's launch shape, and on 16
items of the 64-design multilayer stack batch, for the exact walk and for the fast
(SFU) walk, which is judged only this way.  The tolerance is the one the method
states for R, A and T: max(4 sigma binomial, 1e-4) absolute, sigma of the difference
of the two estimates (plus 2e-5 for the quadrature of the deterministic solver).
"""
import math

import numpy as np
import pytest

from gpu_helpers import gpu_mc, mc_batch_from_media
from paper_2409_00165_gb300 import fos
from paper_2409_00165_gb300 import workloads as W

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

# 0.30 um; the strongly absorbing band; both sides of the k step at 0.4 um (0.3992,
# 0.4048 um); the visible; the near infrared; the long-wavelength end (2.5 um)
PAINT_IDX = [0, 9, 18, 19, 20, 60, 100, 200, 300, 399]


def _tol(p, n1, n2=None):
    var = p * (1 - p) / n1 + (p * (1 - p) / n2 if n2 else 0.0)
    return max(4.0 * math.sqrt(max(var, 0.0)), 1e-4)


@pytest.fixture(autouse=True)
def _reset_tuning():
    fos.fos_mc_set_tuning(0, 0)
    yield
    fos.fos_mc_set_tuning(0, 0)


@pytest.fixture(scope="module")
def paint(orc):
    """The paint layer's inputs (the oracle's Mie), the definition walk at the sampled
    wavelengths and the transfer-equation solution there, computed once."""
    from rte_dom import slab_rat
    m = W.paint_layer()
    props = orc.mie_properties(m["wl"], m["nm"], m["species_group"], m["n_p"], m["radius"],
                               m["vol_frac"], n_groups=m["n_groups"])
    b = mc_batch_from_media(m, props)
    idx = np.array(PAINT_IDX, np.int32)
    n_def = 500000
    ref = orc.mc_run_threads(dict(b, item_list=idx, photons_per_item=n_def, seed=424242))
    dom = [slab_rat(float(props["mu_s"][0, w]), float(props["mu_a"][0, w]),
                    float(props["g"][0, w]), float(m["thickness"][0]),
                    float(m["nm"][0, w].real), n_half=96) for w in idx]
    return dict(m=m, b=b, idx=idx, n_def=n_def, ref=ref, dom=dom)


@pytest.fixture(scope="module")
def stacks(orc):
    m = W.layer_stacks()
    props = orc.mie_properties(m["wl"], m["nm"], m["species_group"], m["n_p"], m["radius"],
                               m["vol_frac"], n_groups=m["n_groups"])
    b = mc_batch_from_media(m, props)
    rng = np.random.default_rng(88)
    items = np.sort(rng.choice(m["n_stacks"] * m["n_wl"], size=16,
                               replace=False)).astype(np.int32)
    n_def = np.minimum(m["n_photons"], 200000)
    ref = orc.mc_run_threads(dict(b, item_list=items, n_photons=n_def, seed=99991))
    return dict(m=m, b=b, items=items, n_def=n_def, ref=ref)


WALKS = [pytest.param(0, id="exact"), pytest.param(fos.FOS_FAST_WALK, id="fast")]


@pytest.mark.parametrize("walk", WALKS)
def test_paint_layer_full_size_vs_definition_and_transfer_equation(paint, walk):
    """All 400 wavelengths x 1e6 photons in the bench's (autotuned) launch shape, exact
    and fast walk; 10 wavelengths compared with the definition walk and the transfer
    equation."""
    m, b, idx = paint["m"], paint["b"], paint["idx"]
    c, _ = gpu_mc(b, flags=fos.FOS_AUTOTUNE | walk)
    N = m["photons_per_item"]
    assert np.all(c[:, :4].sum(axis=1) == N) and np.all(c[:, 3] == 0)
    bad = []
    for r, w in enumerate(idx):
        gpu = c[w, :3] / N
        dfn = paint["ref"][r, :3] / paint["n_def"]
        dom = paint["dom"][r]
        for k in range(3):
            p = 0.5 * (gpu[k] + dfn[k])
            if abs(gpu[k] - dfn[k]) > _tol(p, N, paint["n_def"]):
                bad.append(("definition", int(w), k, gpu[k], dfn[k]))
            if abs(gpu[k] - dom[k]) > _tol(dom[k], N) + 2e-5:
                bad.append(("transfer equation", int(w), k, gpu[k], dom[k]))
    assert not bad, bad


@pytest.mark.parametrize("walk", WALKS)
def test_layer_stacks_items_vs_definition(stacks, walk):
    """16 seeded items of the 64-design x 200-wavelength stack batch (1-3 particle
    layers of different indices on a 5 % reflector), GPU counts at each item's own
    budget from the full batch in the bench's launch shape, against the definition walk
    at min(budget, 2e5) photons."""
    m, b, items, n_def = stacks["m"], stacks["b"], stacks["items"], stacks["n_def"]
    c, _ = gpu_mc(b, flags=fos.FOS_AUTOTUNE | walk)
    assert np.array_equal(c[:, :4].sum(axis=1), m["n_photons"])
    bad = []
    for r, it in enumerate(items):
        n1, n2 = int(m["n_photons"][it]), int(n_def[it])
        for k in range(3):
            f1, f2 = c[it, k] / n1, stacks["ref"][r, k] / n2
            if abs(f1 - f2) > _tol(0.5 * (f1 + f2), n1, n2):
                bad.append((int(it), k, f1, f2))
    assert not bad, bad
