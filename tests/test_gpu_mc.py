"""Parity of the CUDA photon walk (through the C-ABI) with the CPU oracle.

The GPU walk and the oracle's FP32 mirror perform the same IEEE operations in the
same order on the same Philox stream, so counts and per-photon logs must be equal
bit for bit, on every case (index-matched or not).  Statistical bounds vs closed
forms are checked in addition.
"""
import math

import numpy as np
import pytest

from gpu_helpers import gpu_mc, gpu_mie, mc_batch_from_media
from paper_2409_00165_gb300 import fos
from paper_2409_00165_gb300 import workloads as W

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(autouse=True)
def _reset_tuning():
    fos.fos_mc_set_tuning(0, 0)
    yield
    fos.fos_mc_set_tuning(0, 0)


def _slab(ms, ma, g, n, d, N, na=1.0, nb=1.0, sub=None, seed=1, **kw):
    L = len(ms)
    b = dict(n_stacks=1, n_wl=1, max_layers=L, n_layers=np.array([L], np.int32),
             mu_s=np.array(ms, float), mu_a=np.array(ma, float), g=np.array(g, float),
             n_layer=np.array(n, float), thickness=np.array(d, float),
             n_above=np.array([na]), n_below=np.array([nb]), photons_per_item=int(N),
             seed=seed)
    if sub is not None:
        b["substrate_R"] = np.array([sub])
    b.update(kw)
    return b


# ---------------------------------------------------------------- building blocks
def test_philox_bit_exact(orc):
    rng = np.random.default_rng(0)
    ctr = rng.integers(0, 2 ** 32, size=(4096, 4), dtype=np.uint64).astype(np.uint32)
    key = (0x12345678, 0x9ABCDEF0)
    t_ctr = torch.as_tensor(ctr.view(np.int32), device="cuda")
    out = torch.zeros_like(t_ctr)
    fos.check(fos.fos_philox4x32_10(t_ctr, key[0], key[1], out), "philox")
    got = out.cpu().numpy().view(np.uint32)
    for i in range(0, 4096, 97):
        assert np.array_equal(got[i], orc.philox4x32_10(ctr[i], key))
    # cuRAND's device Philox4x32-10 on the same counters and key (a library routine)
    ref = torch.zeros_like(t_ctr)
    fos.check(fos.fos_philox4x32_10(t_ctr, key[0], key[1], ref, curand=True), "curand philox")
    assert torch.equal(ref, out)
    # known-answer vector
    z = torch.zeros((1, 4), dtype=torch.int32, device="cuda")
    o = torch.zeros_like(z)
    fos.fos_philox4x32_10(z, 0, 0, o)
    assert [int(v) for v in o.cpu().numpy().view(np.uint32)[0]] == \
        [0x6627e8d5, 0xe169c58d, 0xbc57ac4c, 0x9b00dbd8]


def test_walk_math_bit_exact_all_inputs(orc):
    k = np.arange(2 ** 23, dtype=np.uint64)
    u = ((2 * k + 1).astype(np.float64) * 2.0 ** -24).astype(np.float32)
    tu = torch.as_tensor(u, device="cuda")
    nl = torch.empty_like(tu)
    cs = torch.empty_like(tu)
    fos.check(fos.fos_walk_math_f32(tu, nl, cs), "walk_math")
    assert np.array_equal(nl.cpu().numpy().view(np.uint32), orc.neg_log_f32(u).view(np.uint32))
    assert np.array_equal(cs.cpu().numpy().view(np.uint32), orc.cos2pi_f32(u).view(np.uint32))


# ---------------------------------------------------------------- photon-for-photon parity
PARITY_CASES = {
    "single_slab": _slab([10.0], [0.1], [0.7], [1.5], [0.5], 100000),
    "index_matched": _slab([6.0], [0.4], [0.8], [1.33], [0.7], 60000, 1.33, 1.33),
    "beer_lambert": _slab([0.0], [0.1], [0.0], [1.5], [0.5], 50000, 1.5, 1.5),
    "iso_unequal": _slab([4.0], [1.0], [0.0], [1.4], [0.8], 50000, 1.0, 1.6),
    "backward_g": _slab([3.0], [0.3], [-0.5], [1.2], [1.0], 50000, 1.0, 1.0),
    "three_layers_sub": _slab([5.0, 0.0, 20.0], [0.2, 0.05, 1.0], [0.6, 0.0, 0.9],
                              [1.5, 1.3, 2.0], [0.3, 0.2, 0.1], 40000, sub=0.3),
    "eight_layers": _slab([1.0, 2, 3, 4, 5, 6, 7, 8], [0.1] * 8,
                          [0.1, 0.2, 0.3, 0.4, 0.5, 0.6, 0.7, 0.8],
                          [1.1, 1.2, 1.3, 1.4, 1.5, 1.6, 1.7, 1.8], [0.1] * 8, 20000),
}


@pytest.mark.parametrize("name", list(PARITY_CASES))
def test_photon_for_photon(orc, name):
    b = PARITY_CASES[name]
    c_gpu, log_gpu, _ = gpu_mc(b, photon_log=True)
    c_orc, log_orc = orc.mc_run(b, fp32=True, photon_log=True)
    assert np.array_equal(log_gpu, log_orc)
    assert np.array_equal(c_gpu, c_orc)
    N = int(b["photons_per_item"])
    assert c_gpu[0, :4].sum() == N


def test_ragged_multi_item_batch(orc):
    """37 items, ragged photon budgets (not multiples of the unit), several layers."""
    rng = np.random.default_rng(7)
    n_st, n_wl, L = 37, 1, 3
    b = dict(n_stacks=n_st, n_wl=n_wl, max_layers=L,
             n_layers=rng.integers(1, L + 1, size=n_st).astype(np.int32),
             mu_s=rng.uniform(0, 20, size=n_st * L), mu_a=rng.uniform(0, 2, size=n_st * L),
             g=rng.uniform(-0.5, 0.95, size=n_st * L), n_layer=rng.uniform(1.0, 2.0, size=n_st * L),
             thickness=rng.uniform(0.05, 0.5, size=n_st * L),
             n_above=rng.uniform(1.0, 1.4, size=n_st), n_below=rng.uniform(1.0, 1.6, size=n_st),
             n_photons=rng.integers(0, 3000, size=n_st).astype(np.int64), seed=12345)
    b["n_photons"][5] = 0
    b["n_photons"][6] = 1
    for tuning in [(0, 0), (64, 1), (128, 32), (96, 3), (32, 5), (256, 7), (160, 2)]:
        fos.fos_mc_set_tuning(*tuning)
        c_gpu, _ = gpu_mc(b)
        c_orc = orc.mc_run(b, fp32=True)
        assert np.array_equal(c_gpu, c_orc), tuning
    assert np.array_equal(c_gpu[:, :4].sum(axis=1), b["n_photons"])


def test_stacks_with_reflector_and_item_list(orc):
    m = W.layer_stacks(n_designs=6, n_wl=9, seed=3, photons_lo=200, photons_hi=2000)
    props = orc.mie_properties(m["wl"], m["nm"], m["species_group"], m["n_p"], m["radius"],
                               m["vol_frac"], n_groups=m["n_groups"])
    b = mc_batch_from_media(m, props)
    c_gpu, _ = gpu_mc(b)
    c_orc = orc.mc_run(b, fp32=True)
    assert np.array_equal(c_gpu, c_orc)
    b2 = dict(b)
    b2["item_list"] = np.array([53, 0, 17, 17, 8], np.int32)
    c2, _ = gpu_mc(b2)
    assert np.array_equal(c2, c_orc[[53, 0, 17, 17, 8]])


def test_sharding_photon_ranges_exact(orc):
    b = _slab([10.0], [0.1], [0.7], [1.5], [0.5], 30000)
    full, _ = gpu_mc(b)
    parts = np.zeros_like(full)
    for first, cnt in [(0, 10000), (10000, 7), (10007, 19993)]:
        bb = dict(b)
        bb["photons_per_item"] = cnt
        bb["photon_first"] = np.array([first], np.int64)
        parts += gpu_mc(bb)[0]
    assert np.array_equal(full, parts)


def test_graph_and_direct_launch_agree():
    b = _slab([10.0], [0.1], [0.7], [1.5], [0.5], 20000)
    a, _ = gpu_mc(b)
    c, _ = gpu_mc(b, flags=fos.FOS_NO_GRAPH)
    d, _ = gpu_mc(b)   # graph replay
    assert np.array_equal(a, c) and np.array_equal(a, d)


# ---------------------------------------------------------------- closed forms at larger N
def test_closed_forms_on_gpu():
    N = 2000000
    c, _ = gpu_mc(_slab([0.0], [0.1], [0.0], [1.5], [0.5], N))
    r, tau = 0.04, math.exp(-0.05)
    R = r + (1 - r) ** 2 * r * tau ** 2 / (1 - r * r * tau * tau)
    T = (1 - r) ** 2 * tau / (1 - r * r * tau * tau)
    for k, p in ((0, R), (2, T), (1, 1 - R - T)):
        assert abs(c[0, k] / N - p) < 4 * math.sqrt(p * (1 - p) / N)
    c, _ = gpu_mc(_slab([0.0], [0.1], [0.0], [1.0], [0.5], N))
    assert c[0, 0] == 0
    p = math.exp(-0.05)
    assert abs(c[0, 2] / N - p) < 4 * math.sqrt(p * (1 - p) / N)


def test_scattering_slab_vs_discrete_ordinates():
    from rte_dom import slab_rat
    N = 4000000
    c, _ = gpu_mc(_slab([10.0], [0.1], [0.7], [1.5], [0.5], N, seed=77))
    ref = slab_rat(10.0, 0.1, 0.7, 0.5, 1.5, n_half=96)
    for k in range(3):
        f = c[0, k] / N
        assert abs(f - ref[k]) < 4 * math.sqrt(ref[k] * (1 - ref[k]) / N) + 2e-4


# ---------------------------------------------------------------- edge cases and errors
def test_empty_and_zero_photons():
    b = _slab([1.0], [0.1], [0.5], [1.5], [0.5], 0)
    c, _ = gpu_mc(b)
    assert np.all(c == 0)
    b2 = dict(b)
    b2["item_list"] = np.zeros(0, np.int32)
    b2["photons_per_item"] = 10
    c2, _ = gpu_mc(b2)
    assert c2.shape[0] == 0


def test_invalid_values_are_reported():
    for bad in (dict(mu_s=np.array([np.nan])), dict(mu_a=np.array([-1.0])),
                dict(g=np.array([1.0])), dict(thickness=np.array([0.0])),
                dict(n_layer=np.array([-1.5])), dict(substrate_R=np.array([1.5])),
                # photon ids are 32-bit: a count of 2^32 (or first + count > 2^32) is refused
                dict(n_photons=np.array([2 ** 32], np.int64)),
                dict(photon_first=np.array([2 ** 32 - 50], np.int64))):
        b = _slab([1.0], [0.1], [0.5], [1.5], [0.5], 100)
        b.update(bad)
        c, st = gpu_mc(b, allow=(fos.FOS_ERR_INVALID_ARG,))
        assert st == fos.FOS_ERR_INVALID_ARG
        assert np.all(c == 0)


def test_injected_failure_and_async_status():
    b = _slab([1.0], [0.1], [0.5], [1.5], [0.5], 1000)
    _, st = gpu_mc(b, flags=fos.FOS_TEST_INJECT, allow=(fos.FOS_ERR_INJECTED,))
    assert st == fos.FOS_ERR_INJECTED
    _, st = gpu_mc(b, flags=fos.FOS_TEST_INJECT | fos.FOS_ASYNC)
    assert st == fos.FOS_OK
    assert fos.fos_sync_status(None, 10000) == fos.FOS_ERR_INJECTED
    assert fos.fos_sync_status(None, 10000) == fos.FOS_OK
    c, st = gpu_mc(b)
    assert st == fos.FOS_OK and c[0, :4].sum() == 1000


def test_runaway_cap(orc):
    b = _slab([50.0], [0.0], [0.9], [1.5], [2.0], 3000, max_events=25)
    c, st = gpu_mc(b, allow=(fos.FOS_ERR_STEP_LIMIT,))
    assert st == fos.FOS_ERR_STEP_LIMIT
    assert np.array_equal(c, orc.mc_run(b, fp32=True))
    assert c[0, 3] > 0 and c[0, :4].sum() == 3000


def test_autotune_picks_a_valid_shape():
    b = _slab([10.0], [0.1], [0.7], [1.5], [0.5], 50000)
    c0, _ = gpu_mc(b)
    c1, _ = gpu_mc(b, flags=fos.FOS_AUTOTUNE)
    assert np.array_equal(c0, c1)


# ---------------------------------------------------------------- full-size paint layer
def test_paint_layer_full_size_sampled_photons(orc):
    """The 400-wavelength, 1e6-photon paint layer in the benchmark's launch shape:
    every item conserves photons exactly, and sampled photons match the oracle."""
    m = W.paint_layer()
    props = orc.mie_properties(m["wl"], m["nm"], m["species_group"], m["n_p"], m["radius"],
                               m["vol_frac"], n_groups=m["n_groups"])
    b = mc_batch_from_media(m, props)
    c, log, _ = gpu_mc(b, photon_log=True, flags=fos.FOS_AUTOTUNE)
    N = m["photons_per_item"]
    assert np.all(c[:, :4].sum(axis=1) == N)
    assert np.all(c[:, 3] == 0)
    rng = np.random.default_rng(2024)
    for _ in range(60):
        w = int(rng.integers(0, m["n_wl"]))
        p = int(rng.integers(0, N))
        one = dict(b)
        one["item_list"] = np.array([w], np.int32)
        one["photons_per_item"] = 1
        one["photon_first"] = np.full(m["n_wl"], p, np.int64)
        _, lo = orc.mc_run(one, fp32=True, photon_log=True)
        assert log[w, p] == lo[0, 0], (w, p)


def test_host_wait_is_bounded():
    """fos_sync_status with a 1 ms limit on a stream still running a long walk returns
    FOS_ERR_TIMEOUT at once; a later wait returns the real status."""
    b = _slab([20.0], [0.01], [0.9], [1.5], [5.0], 20000000)
    from gpu_helpers import to_dev
    f64 = torch.float64
    keep = {k: to_dev(b[k], f64) for k in ("mu_s", "mu_a", "g", "n_layer", "thickness",
                                            "n_above", "n_below")}
    bb = fos.make_batch(1, 1, 1, photons_per_item=b["photons_per_item"], seed=3, **keep)
    counts = torch.zeros((1, fos.FOS_NCOUNT), dtype=torch.int64, device="cuda")
    assert fos.fos_mc_spectrum(bb, counts, None, 0, fos.FOS_ASYNC) == fos.FOS_OK
    assert fos.fos_sync_status(None, 1) == fos.FOS_ERR_TIMEOUT
    assert fos.fos_sync_status(None, 600000) == fos.FOS_OK
    assert int(counts[0, :4].sum()) == 20000000


def test_batch_keeps_temporary_tensors_alive(orc):
    """make_batch holds its tensors: a batch built from temporaries still reads them after
    the caching allocator has handed out new blocks of the same size."""
    ref = W.single_slab(n_photons=3000)
    t = lambda v: torch.as_tensor(np.asarray(v, np.float64), device="cuda")
    b = fos.make_batch(1, 1, 1, t(ref["mu_s"]), t(ref["mu_a"]), t(ref["g"]), t(ref["n_layer"]),
                       t(ref["thickness"]), photons_per_item=3000, seed=ref["seed"])
    junk = [torch.zeros(1, dtype=torch.float64, device="cuda") for _ in range(16)]
    counts = torch.zeros((1, fos.FOS_NCOUNT), dtype=torch.int64, device="cuda")
    fos.check(fos.fos_mc_spectrum(b, counts), "temporaries")
    assert np.array_equal(counts.cpu().numpy(), orc.mc_run(ref, fp32=True))
    del junk


def test_layer_stacks_full_size_sampled_photons(orc):
    """The 64-design x 200-wavelength uneven stack batch (log-uniform 1e4-1e6 photons per
    item, reflector below) in the bench's autotuned launch shape: every item conserves
    its photons.  Then 12 sampled items run again with per-photon logs (same counts: the
    walk does not depend on the launch shape), and 60 sampled photons match the oracle's
    one-photon walks."""
    m = W.layer_stacks()
    props = orc.mie_properties(m["wl"], m["nm"], m["species_group"], m["n_p"], m["radius"],
                               m["vol_frac"], n_groups=m["n_groups"])
    b = mc_batch_from_media(m, props)
    c, _ = gpu_mc(b, flags=fos.FOS_AUTOTUNE)
    assert np.array_equal(c[:, :4].sum(axis=1), m["n_photons"])
    assert np.all(c[:, 3] == 0)
    rng = np.random.default_rng(77)
    items = np.sort(rng.choice(m["n_stacks"] * m["n_wl"], size=12, replace=False)).astype(np.int32)
    bl = dict(b, item_list=items)
    c2, log, _ = gpu_mc(bl, photon_log=True)
    assert np.array_equal(c2, c[items])
    for _ in range(60):
        k = int(rng.integers(0, len(items)))
        it = int(items[k])
        p = int(rng.integers(0, m["n_photons"][it]))
        one = dict(b)
        one["item_list"] = np.array([it], np.int32)
        one["n_photons"] = np.ones_like(m["n_photons"])
        one["photon_first"] = np.full(len(m["n_photons"]), p, np.int64)
        _, lo = orc.mc_run(one, fp32=True, photon_log=True)
        assert log[k, p] == lo[0, 0], (it, p)
