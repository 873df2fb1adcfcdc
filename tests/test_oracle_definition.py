"""Pins of the oracle's definition walk (section "Photon transport", written in the
order the section describes it, FP64, with its own sequential random stream), and the
statistical agreement of the fast walk's operation order with it.

The definition is pinned to closed forms (Beer-Lambert, the incoherent Fresnel slab,
an opaque reflector, incoherent adding, oblique incidence, a conductor below),
invariants, and the discrete-ordinates solution of the transfer equation
(`rte_dom.slab_rat`, an independent deterministic method), including slabs at the
optical depths of the 300 um paint layer (tau_d from 17 to 456).

The fast walk (the GPU kernel, mirrored bit for bit by the oracle's FP32 mode) differs
from the definition in ways that are exact in real arithmetic: reciprocals of mu_t and
2g in place of divisions, the collision test tau |mu| < mu_t dist in place of
tau / mu_t < dist / |mu|, the carried optical depth clamped at 0, one Horner chain for
cos(2 pi u), a 2^-23 uniform grid, and a random layout with the entry draw on word 3 of
collision block 0.  The tests at the end check that these leave R, A and T unchanged
within binomial noise, in both the FP32 mirror and the same order in FP64.
"""
import math
import os

import numpy as np
import pytest

from rte_dom import slab_rat
from paper_2409_00165_gb300 import workloads as W

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _mode(orc):
    return orc.MODE_DEFINITION


def _batch(mu_s, mu_a, g, n, d, N, n_above=1.0, n_below=1.0, sub=None, seed=31, **kw):
    L = len(mu_s)
    b = dict(n_stacks=1, n_wl=1, max_layers=L, n_layers=np.array([L], np.int32),
             mu_s=np.array(mu_s, float), mu_a=np.array(mu_a, float), g=np.array(g, float),
             n_layer=np.array(n, float), thickness=np.array(d, float),
             n_above=np.array([n_above]), n_below=np.array([n_below]),
             photons_per_item=int(N), seed=seed)
    if sub is not None:
        b["substrate_R"] = np.array([sub])
    b.update(kw)
    return b


def _ok(count, N, p, k=4.0, extra=0.0):
    s = math.sqrt(max(p * (1 - p), 1e-12) / N)
    return abs(count / N - p) <= k * s + extra


def _run(orc, b, threads=0, mode=None):
    return orc.mc_run_threads(b, mode=orc.MODE_DEFINITION if mode is None else mode,
                              threads=threads)


# ---------------------------------------------------------------- closed forms
def test_definition_beer_lambert(orc):
    N = 200000
    for n, c0 in ((1.0, 1.0), (1.5, 1.0), (1.0, 0.5)):
        b = _batch([0.0], [0.1], [0.0], [n], [0.5], N, n, n, cos_incidence=np.array([c0]))
        c = _run(orc, b)[0]
        assert c[0] == 0 and c[3] == 0 and c[:4].sum() == N
        assert _ok(c[2], N, math.exp(-0.05 / c0))


def test_definition_fresnel_slab_golden(orc):
    vals = {}
    with open(os.path.join(GOLDEN, "fresnel_slab.txt")) as fh:
        for line in fh:
            if line.strip() and not line.startswith("#"):
                k, v = line.split()
                vals[k] = float(v)
    N = 400000
    c = _run(orc, _batch([0.0], [0.1], [0.0], [1.5], [0.5], N))[0]
    assert _ok(c[0], N, vals["R"]) and _ok(c[1], N, vals["A"]) and _ok(c[2], N, vals["T"])


@pytest.mark.parametrize("c0", [0.9, 0.4])
def test_definition_oblique_slab_and_conductor(orc, c0):
    mu_a, d, n = 0.4, 1.0, 1.5
    N = 300000
    r, ct = orc.fresnel(1.0, n, c0)
    tau = math.exp(-mu_a * d / ct)
    R = r + (1 - r) ** 2 * r * tau ** 2 / (1 - r * r * tau * tau)
    T = (1 - r) ** 2 * tau / (1 - r * r * tau * tau)
    c = _run(orc, _batch([0.0], [mu_a], [0.0], [n], [d], N, cos_incidence=np.array([c0])))[0]
    assert _ok(c[0], N, R) and _ok(c[2], N, T)
    # a conductor n + ik below: what it does not reflect is transmitted into it
    nc, kc = 1.2, 7.0
    Rc = orc.fresnel_conductor(n, nc, kc, ct)
    den = 1 - r * Rc * tau * tau
    R = r + (1 - r) ** 2 * Rc * tau * tau / den
    T = (1 - r) * tau * (1 - Rc) / den
    b = _batch([0.0], [mu_a], [0.0], [n], [d], N, n_below=nc, cos_incidence=np.array([c0]),
               k_below=np.array([kc]))
    c = _run(orc, b)[0]
    assert _ok(c[0], N, R) and _ok(c[2], N, T)


def test_definition_reflector_and_adding(orc):
    r, Rs = 0.04, 0.35
    tau = math.exp(-0.3 * 0.5)
    R = r + (1 - r) ** 2 * Rs * tau ** 2 / (1 - r * Rs * tau ** 2)
    T = (1 - r) * tau * (1 - Rs) / (1 - r * Rs * tau ** 2)
    N = 300000
    c = _run(orc, _batch([0.0], [0.3], [0.0], [1.5], [0.5], N, sub=Rs))[0]
    assert _ok(c[0], N, R) and _ok(c[2], N, T)
    # two absorbing layers of different index, unequal media: incoherent adding
    def iface(a, b):
        q = ((a - b) / (a + b)) ** 2
        return (q, 1 - q, q, 1 - q)

    def layer(ma, d):
        t = math.exp(-ma * d)
        return (0.0, t, 0.0, t)

    el = [iface(1.0, 1.5), layer(0.3, 0.4), iface(1.5, 2.0), layer(0.8, 0.25), iface(2.0, 1.2)]
    Rf, Tf, Rb, Tb = el[0]
    for (R2f, T2f, R2b, T2b) in el[1:]:
        den = 1 - Rb * R2f
        Rf, Tf, Rb, Tb = (Rf + Tf * Tb * R2f / den, Tf * T2f / den,
                          R2b + T2b * T2f * Rb / den, T2b * Tb / den)
    c = _run(orc, _batch([0, 0], [0.3, 0.8], [0, 0], [1.5, 2.0], [0.4, 0.25], N, 1.0, 1.2))[0]
    assert _ok(c[0], N, Rf) and _ok(c[2], N, Tf)


def test_definition_entry_total_reflection(orc):
    b = _batch([1.0], [0.5], [0.0], [1.0], [1.0], 3000, n_above=1.5,
               cos_incidence=np.array([0.5]))
    c = _run(orc, b)[0]
    assert c[0] == 3000 and c[4] == 0 and c[5] == 0


# ---------------------------------------------------------------- invariants
def test_definition_invariants(orc):
    N = 20000
    b = _batch([5.0, 2.0], [0.0, 0.0], [0.8, -0.2], [1.4, 1.7], [0.3, 0.6], N, 1.0, 1.3)
    c = orc.mc_run(b, mode=orc.MODE_DEFINITION)[0]
    assert c[1] == 0 and c[3] == 0 and c[:4].sum() == N
    # shards by photon range sum to the single run exactly
    assert np.array_equal(_run(orc, b, threads=3)[0], c)
    # the event cap
    b = _batch([50.0], [0.0], [0.9], [1.5], [2.0], 2000, max_events=30)
    c = orc.mc_run(b, mode=orc.MODE_DEFINITION)[0]
    assert c[3] > 0 and c[:4].sum() == 2000 and c[4] + c[5] <= 30 * 2000


def test_definition_carry_over_across_identical_sublayers(orc):
    """Splitting a layer in two identical halves changes nothing (carry-over of the
    unused optical depth at an internal boundary with no index step)."""
    N = 200000
    one = _run(orc, _batch([4.0], [0.5], [0.6], [1.4], [0.6], N))[0]
    two = _run(orc, _batch([4.0, 4.0], [0.5, 0.5], [0.6, 0.6], [1.4, 1.4], [0.2, 0.4], N,
                           seed=99))[0]
    for k in range(3):
        p = one[k] / N
        assert abs(two[k] / N - p) <= 4 * math.sqrt(2 * p * (1 - p) / N) + 1e-12


# ---------------------------------------------------------------- transfer equation
def _paint_layer_slabs(orc, idx):
    m = W.paint_layer()
    p = orc.mie_properties(m["wl"], m["nm"], m["species_group"], m["n_p"], m["radius"],
                           m["vol_frac"])
    out = []
    for i in idx:
        out.append((float(p["mu_s"][0, i]), float(p["mu_a"][0, i]), float(p["g"][0, i]),
                    float(m["thickness"][0]), float(m["nm"][0, i].real)))
    return out


DOM_CASES = [
    # mu_s, mu_a, g, d, n_in, n_above, n_below, mu0, photons
    (10.0, 0.1, 0.7, 0.5, 1.5, 1.0, 1.0, 1.0, 600000),   # the single-slab workload
    (3.0, 0.3, -0.5, 1.0, 1.33, 1.33, 1.33, 1.0, 300000),  # back-scattering, index matched
    (4.0, 1.0, 0.0, 0.8, 1.4, 1.0, 1.6, 1.0, 300000),     # isotropic, unequal boundaries
    (10.0, 0.1, 0.7, 0.5, 1.5, 1.0, 1.0, 0.5, 300000),    # oblique beam
]


@pytest.mark.parametrize("case", DOM_CASES)
def test_definition_vs_discrete_ordinates(orc, case):
    ms, ma, g, d, n, na, nb, mu0, N = case
    ref = slab_rat(ms, ma, g, d, n, na, nb, n_half=96, mu0=mu0)
    b = _batch([ms], [ma], [g], [n], [d], N, na, nb, cos_incidence=np.array([mu0]))
    c = _run(orc, b)[0]
    for k in range(3):
        assert _ok(c[k], N, ref[k], 4.0, 2e-4), (k, c[k] / N, ref[k])


@pytest.mark.slow
def test_definition_vs_discrete_ordinates_paint_layer_depths(orc):
    """The paint layer's own optical depths (tau_d = 17, 44, 244 at 2.5, 1.95 and
    0.41 um; albedo up to 0.9986): the regime of the benchmarked spectrum."""
    N = 100000
    for (ms, ma, g, d, n) in _paint_layer_slabs(orc, [399, 300, 20]):
        ref = slab_rat(ms, ma, g, d, n, n_half=96)
        c = _run(orc, _batch([ms], [ma], [g], [n], [d], N))[0]
        for k in range(3):
            assert _ok(c[k], N, ref[k], 4.0, 2e-4), (ms, k, c[k] / N, ref[k])


# ---------------------------------------------------------------- the fast walk's order
ORDER_CASES = [
    # the single slab; a strongly forward-scattering slab between unequal media; three
    # layers on a reflector; an oblique beam on a conductor; a paint-layer wavelength
    dict(b=_batch([10.0], [0.1], [0.7], [1.5], [0.5], 400000)),
    dict(b=_batch([20.0], [0.05], [0.95], [1.6], [0.3], 200000, 1.0, 1.3)),
    dict(b=_batch([8.0, 0.5, 3.0], [0.2, 0.05, 1.0], [0.8, 0.0, -0.3], [1.45, 1.7, 1.3],
                  [0.2, 0.1, 0.3], 300000, sub=0.4)),
    dict(b=_batch([5.0], [0.5], [0.8], [1.5], [0.5], 300000, n_below=0.96,
                  k_below=np.array([6.69]), cos_incidence=np.array([0.4]))),
]


@pytest.mark.parametrize("case", range(len(ORDER_CASES)))
def test_fast_walk_order_agrees_with_definition(orc, case):
    """Reciprocals, the division-free collision test, the tau clamp, the merged
    cos(2 pi u) chain, the 2^-23 uniforms and the entry draw on word 3 of block 0 leave
    R, A and T unchanged: the FP32 mirror (bit-exact with the GPU walk) and the same
    order in FP64 agree with the definition within 4 sigma of the difference of two
    independent binomial estimates."""
    b = dict(ORDER_CASES[case]["b"])
    N = b["photons_per_item"]
    ref = _run(orc, dict(b, seed=501))[0]
    for mode in (orc.MODE_F32_MIRROR, orc.MODE_F64_ORDER):
        c = _run(orc, dict(b, seed=777), mode=mode)[0]
        assert c[:4].sum() == N
        for k in range(3):
            p = 0.5 * (c[k] + ref[k]) / N
            sig = math.sqrt(max(2 * p * (1 - p) / N, 1e-12))
            assert abs(c[k] - ref[k]) / N <= 4 * sig, (mode, k, c[k] / N, ref[k] / N)
