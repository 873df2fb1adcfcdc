"""GPU parity of the boundary and incidence variants of the walk (oblique incidence, a
conductor below the stack) and of the Eq. 21 solar-weighted totals, through the C ABI.

The walk variants follow the same rule as the rest of the walk: counts and per-photon
logs equal the oracle's FP32 mirror bit for bit.  The totals are FP64 sums in another
order than the oracle's, so they agree to rounding."""
import numpy as np
import pytest

from gpu_helpers import gpu_mc, mc_batch_from_media, to_dev
from paper_2409_00165_gb300 import fos
from paper_2409_00165_gb300 import workloads as W

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def _slab(ms, ma, g, n, d, N, seed=3, **kw):
    L = len(ms)
    b = dict(n_stacks=1, n_wl=1, max_layers=L, n_layers=np.array([L], np.int32),
             mu_s=np.array(ms, float), mu_a=np.array(ma, float), g=np.array(g, float),
             n_layer=np.array(n, float), thickness=np.array(d, float),
             photons_per_item=int(N), seed=seed)
    b.update(kw)
    return b


CASES = {
    "oblique_0.5": _slab([10.0], [0.1], [0.7], [1.5], [0.5], 20000,
                         cos_incidence=np.array([0.5])),
    "oblique_grazing": _slab([3.0], [0.3], [0.2], [1.3], [0.3], 20000,
                             cos_incidence=np.array([0.05])),
    "oblique_index_matched": _slab([4.0], [0.5], [0.5], [1.0], [0.5], 20000,
                                   cos_incidence=np.array([0.7])),
    "entry_total_reflection": _slab([4.0], [0.5], [0.5], [1.0], [0.5], 5000,
                                    cos_incidence=np.array([0.5]), n_above=np.array([1.5])),
    "conductor_normal": _slab([5.0], [0.5], [0.8], [1.5], [0.5], 20000,
                              n_below=np.array([1.2]), k_below=np.array([7.0])),
    "conductor_oblique_3_layers": _slab([5.0, 0.0, 12.0], [0.5, 0.2, 0.1], [0.8, 0.0, -0.3],
                                        [1.5, 1.8, 1.3], [0.2, 0.1, 0.4], 20000,
                                        cos_incidence=np.array([0.6]),
                                        n_below=np.array([0.96]), k_below=np.array([6.69])),
}


@pytest.mark.parametrize("name", list(CASES))
def test_photon_for_photon(orc, name):
    b = CASES[name]
    c_gpu, log_gpu, _ = gpu_mc(b, photon_log=True)
    c_orc, log_orc = orc.mc_run(b, fp32=True, photon_log=True)
    assert np.array_equal(log_gpu, log_orc)
    assert np.array_equal(c_gpu, c_orc)
    assert c_gpu[0, :4].sum() == b["photons_per_item"]


def test_mixed_batch_per_item_incidence_and_boundaries(orc):
    """41 items: per-item incidence cosines, conductors, dielectrics and reflectors mixed,
    ragged budgets, an item list with repeats."""
    rng = np.random.default_rng(31)
    n_st, n_wl, L = 41, 1, 2
    b = dict(n_stacks=n_st, n_wl=n_wl, max_layers=L,
             n_layers=rng.integers(1, L + 1, size=n_st).astype(np.int32),
             mu_s=rng.uniform(0, 15, n_st * L), mu_a=rng.uniform(0, 1.5, n_st * L),
             g=rng.uniform(-0.3, 0.9, n_st * L), n_layer=rng.uniform(1.0, 2.0, n_st * L),
             thickness=rng.uniform(0.05, 0.5, n_st * L),
             n_above=rng.choice([1.0, 1.0, 1.33], n_st), n_below=rng.uniform(0.5, 2.0, n_st),
             k_below=np.where(rng.uniform(size=n_st) < 0.5, rng.uniform(0.1, 8.0, n_st), 0.0),
             cos_incidence=np.where(rng.uniform(size=n_st) < 0.3, 1.0,
                                    rng.uniform(0.02, 1.0, n_st)),
             n_photons=rng.integers(0, 2500, n_st).astype(np.int64), seed=99)
    c_gpu, _ = gpu_mc(b)
    c_orc = orc.mc_run(b, fp32=True)
    assert np.array_equal(c_gpu, c_orc)
    b["item_list"] = np.array([40, 3, 3, 17, 0], np.int32)
    c2, _ = gpu_mc(b)
    assert np.array_equal(c2, c_orc[[40, 3, 3, 17, 0]])


def test_defaults_equal_explicit_normal_dielectric():
    b = _slab([10.0], [0.1], [0.7], [1.5], [0.5], 30000)
    a, _ = gpu_mc(b)
    c, _ = gpu_mc(dict(b, cos_incidence=np.array([1.0]), k_below=np.array([0.0])))
    assert np.array_equal(a, c)


def test_invalid_incidence_and_conductor():
    for bad in (dict(cos_incidence=np.array([0.0])), dict(cos_incidence=np.array([1.5])),
                dict(cos_incidence=np.array([np.nan])), dict(k_below=np.array([-1.0])),
                dict(k_below=np.array([np.inf])),
                dict(k_below=np.array([2.0]), substrate_R=np.array([0.5]))):
        b = _slab([1.0], [0.1], [0.5], [1.5], [0.5], 100)
        b.update(bad)
        c, st = gpu_mc(b, allow=(fos.FOS_ERR_INVALID_ARG,))
        assert st == fos.FOS_ERR_INVALID_ARG
        assert np.all(c == 0)


# ------------------------------------------------------------------ Eq. 21 totals
def _solar(n_stacks, wl, G, counts, allow=(fos.FOS_OK,), flags=0):
    out = torch.full((n_stacks * 3,), -1.0, dtype=torch.float64, device="cuda")
    st = fos.fos_solar_weighted(n_stacks, to_dev(wl, torch.float64), to_dev(G, torch.float64),
                                to_dev(counts, torch.int64), out, flags=flags)
    torch.cuda.synchronize()
    fos.check(st, "fos_solar_weighted", allow)
    return out.cpu().numpy().reshape(n_stacks, 3), st


def test_solar_weighted_matches_oracle(orc):
    rng = np.random.default_rng(8)
    for n_stacks, n_wl in ((37, 301), (3, 2), (5, 1), (2, 1000)):
        wl = np.sort(rng.uniform(0.3, 2.5, n_wl)) if n_wl > 2 else np.linspace(0.3, 2.5, n_wl)
        wl = np.unique(wl)
        n_wl = wl.size
        G = W.solar_like_irradiance(wl)
        c = np.zeros((n_stacks * n_wl, 6), np.int64)
        c[:, :3] = rng.integers(0, 10 ** 6, (n_stacks * n_wl, 3))
        c[0, :3] = 0   # an empty item: fractions 0
        got, _ = _solar(n_stacks, wl, G, c)
        want = orc.solar_weighted(c, wl, G, n_stacks)
        assert np.allclose(got, want, rtol=1e-12, atol=1e-15)


def test_solar_weighted_errors():
    wl = np.array([0.5, 1.0, 0.9])
    c = np.ones((3, 6), np.int64)
    _, st = _solar(1, wl, np.ones(3), c, allow=(fos.FOS_ERR_INVALID_ARG,))
    assert st == fos.FOS_ERR_INVALID_ARG
    wl = np.array([0.5, 1.0, 1.5])
    for G in (np.array([1.0, -1.0, 1.0]), np.zeros(3), np.array([1.0, np.nan, 1.0])):
        _, st = _solar(1, wl, G, c, allow=(fos.FOS_ERR_INVALID_ARG,))
        assert st == fos.FOS_ERR_INVALID_ARG
    _, st = _solar(1, wl, np.ones(3), c, allow=(fos.FOS_ERR_INJECTED,),
                   flags=fos.FOS_TEST_INJECT)
    assert st == fos.FOS_ERR_INJECTED


def test_oblique_conductor_full_size_sampled_photons(orc):
    """The bench's oblique-incidence leg at full size: the paint-layer medium, 50 um thick,
    on the aluminium-like metal at 0, 30 and 60 degrees, 400 wavelengths x 1e6 photons.
    Every item conserves its photons; 8 logged items give 40 sampled photons that match
    the oracle's one-photon walks."""
    m = W.oblique_conductor_media()
    props = orc.mie_properties(m["wl"], m["nm"], m["species_group"], m["n_p"], m["radius"],
                               m["vol_frac"], n_groups=m["n_groups"])
    b = mc_batch_from_media(m, props, photons=1000000)
    b.update(cos_incidence=m["cos_incidence"], n_below=m["n_below"], k_below=m["k_below"],
             seed=13)
    c, _ = gpu_mc(b, flags=fos.FOS_AUTOTUNE)
    assert np.all(c[:, :4].sum(axis=1) == 1000000)
    rng = np.random.default_rng(5)
    items = np.sort(rng.choice(len(m["cos_incidence"]), size=8, replace=False)).astype(np.int32)
    c2, log, _ = gpu_mc(dict(b, item_list=items), photon_log=True)
    assert np.array_equal(c2, c[items])
    for _ in range(40):
        k = int(rng.integers(0, len(items)))
        it = int(items[k])
        p = int(rng.integers(0, 1000000))
        one = dict(b, item_list=np.array([it], np.int32), photons_per_item=1,
                   photon_first=np.full(len(m["cos_incidence"]), p, np.int64))
        _, lo = orc.mc_run(one, fp32=True, photon_log=True)
        assert log[k, p] == lo[0, 0], (it, p)
