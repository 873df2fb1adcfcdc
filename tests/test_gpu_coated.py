"""Parity of the FP64 CUDA core-shell Mie path (supplement Eqs. S1-S9) with the CPU
oracle, through fos_mie_properties_cs."""
import numpy as np
import pytest

from gpu_helpers import gpu_mie
from paper_2409_00165_gb300 import fos
from paper_2409_00165_gb300 import workloads as W

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

RTOL = 1e-10   # FP64 kernel vs FP64 oracle: same equations, different recurrences


def _oracle(orc, m):
    return orc.mie_properties(m["wl"], m["nm"], m["species_group"], m["n_p"], m["radius"],
                              m["vol_frac"], n_groups=m["n_groups"],
                              core_radius=m["core_radius"], n_core=m["n_core"])


def _close(a, b, rtol=RTOL, atol=0.0):
    a, b = np.asarray(a), np.asarray(b)
    return np.all(np.abs(a - b) <= rtol * np.abs(b) + atol)


def test_hollow_silica_400_wavelengths(orc):
    m = W.hollow_silica_media()
    g, o = gpu_mie(m), _oracle(orc, m)
    for k in ("mu_s", "g", "q_ext", "q_sca"):
        assert _close(g[k], o[k]), k
    assert _close(g["g_species"], o["g_sp"])
    # mu_a of weakly absorbing silica in air is C(Q_ext - Q_sca) (Eqs. 13-14): a difference
    # of two O(1) efficiencies, so its rounding error scales with the extinction
    assert _close(g["mu_a"], o["mu_a"], atol=RTOL * (o["mu_s"] + o["mu_a"]))
    # a hollow sphere scatters less than the solid one of the same outer size in the IR
    assert np.all(g["mu_s"][:3, -50:] < g["mu_s"][3:, -50:])


def test_mixed_species_edge_cases(orc):
    rng = np.random.default_rng(5)
    wl = np.array([0.3, 0.45, 0.8, 1.6, 2.5])
    #            b      a        kind
    shapes = [(0.35, 0.25), (0.3, 0.1), (0.55, 0.4), (0.2, 1e-5), (0.5, 0.5 - 1e-7),
              (1.5, 1.2), (0.4, 0.0), (0.05, 0.03), (2.0, 0.5)]
    n_sp = len(shapes)
    ns = (rng.uniform(1.3, 3.0, (n_sp, wl.size))
          + 1j * rng.choice([0.0, 1e-5, 1e-2, 0.3], (n_sp, wl.size)))
    nc = (rng.uniform(1.0, 4.0, (n_sp, wl.size))
          + 1j * rng.choice([0.0, 1e-4, 0.1, 2.0], (n_sp, wl.size)))
    nm = np.array([[1.0 + 0j] * wl.size, [1.33 + 1e-6j] * wl.size, [1.48 + 1e-3j] * wl.size])
    m = dict(wl=wl, nm=nm, n_groups=3,
             species_group=np.array([0, 0, 0, 1, 1, 1, 2, 2, 2], np.int32), n_p=ns, n_core=nc,
             radius=np.array([b for b, _ in shapes]),
             core_radius=np.array([a for _, a in shapes]),
             vol_frac=np.array([0.01, 0.02, 0.05, 0.05, 0.1, 0.01, 0.1, 0.2, 0.05]))
    g, o = gpu_mie(m), _oracle(orc, m)
    for k in ("q_ext", "q_sca", "g_species"):
        ok = "g_sp" if k == "g_species" else k
        assert _close(g[k], o[ok], rtol=1e-9, atol=1e-300), k
    for k in ("mu_s", "mu_a", "g"):
        assert _close(g[k], o[k], rtol=1e-9), k


def test_zero_core_is_the_homogeneous_path():
    """A zero core takes the homogeneous-sphere evaluation.  The core-shell entry runs it
    in another kernel instantiation, whose multiply-add contraction may differ, so the
    two agree to a few ulps rather than bit for bit."""
    m = W.hollow_silica_media(n_wl=37)
    m["core_radius"] = np.zeros_like(m["core_radius"])
    cs = gpu_mie(m)
    plain = {k: v for k, v in m.items() if k not in ("core_radius", "n_core")}
    g = gpu_mie(plain)
    for k in ("mu_s", "g", "q_ext", "q_sca", "g_species"):
        assert np.all(np.abs(cs[k] - g[k]) <= 1e-13 * np.abs(g[k])), k
    # mu_a is a difference of extinction and scattering (Eqs. 13-14): bounded by extinction
    assert np.all(np.abs(cs["mu_a"] - g["mu_a"]) <= 1e-13 * (g["mu_s"] + g["mu_a"]))


def test_invalid_core_radius_and_range():
    m = W.hollow_silica_media(n_wl=8)
    for bad in (m["radius"][0], m["radius"][0] * 1.01, -0.1):
        mm = dict(m, core_radius=m["core_radius"].copy())
        mm["core_radius"][0] = bad
        r = gpu_mie(mm, allow=(fos.FOS_ERR_INVALID_ARG,))
        assert r["status"] == fos.FOS_ERR_INVALID_ARG
    mm = dict(m, radius=m["radius"] * 200, core_radius=m["core_radius"] * 200)
    r = gpu_mie(mm, allow=(fos.FOS_ERR_OUT_OF_RANGE,))
    assert r["status"] == fos.FOS_ERR_OUT_OF_RANGE
