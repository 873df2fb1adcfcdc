"""The fast walk (FOS_FAST_WALK): -ln u and cos 2 pi u on the special-function unit,
approximate reciprocal and square root on the collision path.  It is not bit-exact
with anything, so it is judged statistically: its transcendentals against double-
precision libm over every uniform the walk can draw, its counts against the exact walk
on the same random numbers, and against the transfer equation.  The full-size paint
layer and the stack batch are compared with the definition walk in
test_gpu_definition.py."""
import math

import numpy as np
import pytest

from gpu_helpers import gpu_mc
from paper_2409_00165_gb300 import fos

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(autouse=True)
def _reset_tuning():
    fos.fos_mc_set_tuning(0, 0)
    yield
    fos.fos_mc_set_tuning(0, 0)


def _slab(ms, ma, g, n, d, N, na=1.0, nb=1.0, seed=1, **kw):
    L = len(ms)
    b = dict(n_stacks=1, n_wl=1, max_layers=L, n_layers=np.array([L], np.int32),
             mu_s=np.array(ms, float), mu_a=np.array(ma, float), g=np.array(g, float),
             n_layer=np.array(n, float), thickness=np.array(d, float),
             n_above=np.array([na]), n_below=np.array([nb]), photons_per_item=int(N),
             seed=seed)
    b.update(kw)
    return b


def test_sfu_math_error_on_every_uniform():
    """All 2^23 uniforms (2k+1) 2^-24: -ln u within 2^-21 + 2^-21 |ln u| and cos 2 pi u
    within 2^-19 of double-precision libm."""
    k = np.arange(2 ** 23, dtype=np.uint64)
    u = ((2 * k + 1).astype(np.float64) * 2.0 ** -24).astype(np.float32)
    tu = torch.as_tensor(u, device="cuda")
    nl = torch.empty_like(tu)
    cs = torch.empty_like(tu)
    fos.check(fos.fos_walk_math_f32(tu, nl, cs, fast=True), "walk_math fast")
    ud = u.astype(np.float64)
    ref_nl = -np.log(ud)
    ref_cs = np.cos(2 * np.pi * ud)
    err_nl = np.abs(nl.cpu().numpy().astype(np.float64) - ref_nl)
    err_cs = np.abs(cs.cpu().numpy().astype(np.float64) - ref_cs)
    assert np.all(err_nl <= 2.0 ** -21 * (1 + ref_nl)), err_nl.max()
    assert np.all(err_cs <= 2.0 ** -19), err_cs.max()


def test_fast_walk_tracks_exact_walk():
    """Same random numbers: counts within 4 sigma of a binomial difference, and
    conservation exact, on single and layered cases."""
    cases = [
        _slab([10.0], [0.1], [0.7], [1.5], [0.5], 2000000),
        _slab([5.0, 0.0, 20.0], [0.2, 0.05, 1.0], [0.6, 0.0, 0.9], [1.5, 1.3, 2.0],
              [0.3, 0.2, 0.1], 1000000, substrate_R=np.array([0.3])),
        _slab([5.0], [0.5], [0.8], [1.5], [0.5], 1000000, nb=1.2, k_below=np.array([7.0]),
              cos_incidence=np.array([0.5])),
    ]
    for b in cases:
        N = b["photons_per_item"]
        ce, _ = gpu_mc(b)
        cf, _ = gpu_mc(b, flags=fos.FOS_FAST_WALK)
        assert cf[0, :4].sum() == N and cf[0, 3] == 0
        for k in range(3):
            p = ce[0, k] / N
            assert abs(cf[0, k] - ce[0, k]) / N <= 4 * math.sqrt(2 * p * (1 - p) / N) + 1e-6


def test_fast_walk_vs_discrete_ordinates():
    from rte_dom import slab_rat
    N = 4000000
    c, _ = gpu_mc(_slab([10.0], [0.1], [0.7], [1.5], [0.5], N, seed=78),
                  flags=fos.FOS_FAST_WALK)
    ref = slab_rat(10.0, 0.1, 0.7, 0.5, 1.5, n_half=96)
    for k in range(3):
        assert abs(c[0, k] / N - ref[k]) < 4 * math.sqrt(ref[k] * (1 - ref[k]) / N) + 2e-5


def test_fast_walk_launch_shapes_and_graphs_agree():
    """The fast walk is still a function of (seed, item, photon) only: every launch shape
    and the graph replay give the same counts."""
    rng = np.random.default_rng(3)
    n_st, L = 29, 2
    b = dict(n_stacks=n_st, n_wl=1, max_layers=L,
             n_layers=rng.integers(1, L + 1, size=n_st).astype(np.int32),
             mu_s=rng.uniform(0, 20, size=n_st * L), mu_a=rng.uniform(0, 2, size=n_st * L),
             g=rng.uniform(-0.5, 0.95, size=n_st * L), n_layer=rng.uniform(1.0, 2.0, size=n_st * L),
             thickness=rng.uniform(0.05, 0.5, size=n_st * L),
             n_photons=rng.integers(0, 5000, size=n_st).astype(np.int64), seed=4321)
    ref = None
    for tuning in [(0, 0), (64, 2), (256, 16), (96, 5)]:
        fos.fos_mc_set_tuning(*tuning)
        c, _ = gpu_mc(b, flags=fos.FOS_FAST_WALK)
        if ref is None:
            ref = c
        assert np.array_equal(c, ref), tuning
    c, _ = gpu_mc(b, flags=fos.FOS_FAST_WALK | fos.FOS_NO_GRAPH)
    assert np.array_equal(c, ref)
    assert np.array_equal(ref[:, :4].sum(axis=1), b["n_photons"])


def test_walk_times_recorded():
    """FOS_RECORD_TIMES: one (start, end) per block of the persistent grid, ends after
    starts, all within the launch."""
    b = _slab([10.0], [0.1], [0.7], [1.5], [0.5], 500000)
    c, _ = gpu_mc(b, flags=fos.FOS_RECORD_TIMES)
    t = fos.fos_mc_walk_times()
    assert t.shape[0] >= torch.cuda.get_device_properties(0).multi_processor_count
    assert np.all(t[:, 1] >= t[:, 0]) and np.all(t[:, 0] > 0)
    assert t[:, 1].max() - t[:, 0].min() < 10_000_000_000
    assert c[0, :4].sum() == 500000
