"""Parity of the FP64 CUDA Mie + effective-medium kernels with the CPU oracle."""
import numpy as np
import pytest

from gpu_helpers import gpu_mie
from paper_2409_00165_gb300 import fos
from paper_2409_00165_gb300 import workloads as W

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

RTOL = 1e-10   # FP64 kernel vs FP64 oracle (different recurrences, same equations)


def _oracle(orc, m):
    return orc.mie_properties(m["wl"], m["nm"], m["species_group"], m["n_p"], m["radius"],
                              m["vol_frac"], n_groups=m["n_groups"])


def _close(a, b, rtol=RTOL, atol=0.0):
    a, b = np.asarray(a), np.asarray(b)
    return np.all(np.abs(a - b) <= rtol * np.abs(b) + atol)


def test_paint_layer_400_wavelengths(orc):
    m = W.paint_layer()
    g, o = gpu_mie(m), _oracle(orc, m)
    for k in ("mu_s", "mu_a", "g", "q_ext", "q_sca"):
        assert _close(g[k], o[k]), k
    assert _close(g["g_species"], o["g_sp"])


def test_layer_stacks_all_species(orc):
    m = W.layer_stacks()
    g, o = gpu_mie(m), _oracle(orc, m)
    # groups without particles (unused layer slots) hold matrix absorption only
    for k in ("mu_s", "mu_a", "g"):
        assert _close(g[k], o[k], atol=1e-300), k
    for k in ("q_ext", "q_sca"):
        assert _close(g[k], o[k]), k


def test_host_argument_across_the_upward_psi_switch(orc):
    """psi_n(x) of the host argument comes from its upward recurrence at every order for
    |x| >= 1.5 and from D_n(x) above |x| below that: spheres on both sides of the switch
    and up to |x| = 300 (the chunked pass for large spheres), with particles nearly
    index-matched (m = 1.01), below the host index, absorbing and strongly absorbing."""
    wl = np.array([1.0])
    nm = np.array([[1.48 + 2e-5j]])
    xs = np.array([1.45, 1.499, 1.5, 1.501, 1.6, 3.0, 10.0, 40.0, 150.0, 300.0])
    idx = [1.495 + 0j, 1.2 + 0j, 2.5 + 1e-4j, 3.5 + 0.5j]
    radius = np.repeat(xs / (2 * np.pi * 1.48), len(idx))
    n_p = np.array([[c] for _ in xs for c in idx])
    n_sp = radius.size
    m = dict(wl=wl, nm=nm, n_groups=1, species_group=np.zeros(n_sp, np.int32), n_p=n_p,
             radius=radius, vol_frac=np.full(n_sp, 0.001))
    g, o = gpu_mie(m), _oracle(orc, m)
    # rel 1e-10, and 1e-9 for the spheres of the chunked pass (|x| >= 150), as for the
    # large spheres below (their sums run over hundreds of orders)
    rtol = np.where(np.repeat(xs, len(idx)) >= 150, 1e-9, RTOL)[:, None]
    for k in ("q_ext", "q_sca", "g_species"):
        ok = "g_sp" if k == "g_species" else k
        a, b = np.asarray(g[k]), np.asarray(o[ok])
        rel = np.abs(a - b) / np.abs(b)
        assert np.all(rel <= rtol), (k, np.argmax(rel / rtol), rel.max())


def test_edge_sizes_and_indices(orc):
    rng = np.random.default_rng(11)
    wl = np.array([0.3, 0.31, 0.5, 1.0, 2.5])
    radius = np.array([1e-3, 0.05, 0.37, 1.0, 2.5, 4.0])
    n_sp = radius.size
    n_p = (rng.uniform(1.05, 3.5, size=(n_sp, wl.size))
           + 1j * rng.choice([0.0, 1e-6, 1e-2, 0.5, 2.0], size=(n_sp, wl.size)))
    nm = np.array([[1.0 + 0j] * wl.size, [1.33 + 1e-7j] * wl.size, [1.48 + 1e-3j] * wl.size])
    m = dict(wl=wl, nm=nm, n_groups=3, species_group=np.array([0, 0, 1, 1, 2, 2], np.int32),
             n_p=n_p, radius=radius, vol_frac=np.array([0.01, 0.02, 0.05, 0.05, 0.1, 0.2]))
    g, o = gpu_mie(m), _oracle(orc, m)
    for k in ("q_ext", "q_sca", "g_species"):
        ok = "g_sp" if k == "g_species" else k
        assert _close(g[k], o[ok], rtol=1e-9, atol=1e-300), k
    for k in ("mu_s", "mu_a", "g"):
        assert _close(g[k], o[k], rtol=1e-9), k


def test_host_at_zero_of_psi0(orc):
    """x = 240 pi (r = 60, lambda = 0.5, n_m = 1): psi_0(x) = sin x = 0, and n_max = 1178,
    summed in three chunks of the scratch's 512 orders; x = 40 pi (r = 10): one chunk."""
    for r in (60.0, 10.0):
        m = dict(wl=np.array([0.5]), nm=np.array([[1.0 + 0j]]), n_groups=1,
                 species_group=np.array([0], np.int32), n_p=np.array([[1.5 + 0.01j]]),
                 radius=np.array([r]), vol_frac=np.array([0.1]))
        g, o = gpu_mie(m), _oracle(orc, m)
        for k in ("q_ext", "q_sca", "g_species"):
            ok = "g_sp" if k == "g_species" else k
            assert _close(g[k], o[ok], rtol=1e-9), (r, k)


def test_large_spheres_any_size(orc):
    """Spheres whose n_max exceeds the scratch (FOS_MIE_MAX_TERMS orders per chunk): the
    paint-layer particle at r = 20 um (n_max 680) and r = 60 um (1945) over the wavelength
    grid's ends, absorbing and not, in the paint matrix."""
    wl = np.array([0.3, 0.5, 2.5])
    radius = np.array([20.0, 60.0])
    n_p = np.array([[2.5 + 0.5j, 2.6 + 1e-4j, 2.508 + 1e-4j]] * 2)
    nm = np.array([[1.48 + 3e-6j, 1.48 + 5e-6j, 1.48 + 2.5e-5j]])
    m = dict(wl=wl, nm=nm, n_groups=1, species_group=np.array([0, 0], np.int32), n_p=n_p,
             radius=radius, vol_frac=np.array([0.05, 0.05]))
    g, o = gpu_mie(m), _oracle(orc, m)
    for k in ("q_ext", "q_sca", "g_species"):
        ok = "g_sp" if k == "g_species" else k
        assert _close(g[k], o[ok], rtol=1e-9), k
    for k in ("mu_s", "mu_a", "g"):
        assert _close(g[k], o[k], rtol=1e-9), k


def test_invalid_and_injected():
    m = W.paint_layer(n_wl=8)
    m["vol_frac"] = np.array([1.2])
    r = gpu_mie(m, allow=(fos.FOS_ERR_INVALID_ARG,))
    assert r["status"] == fos.FOS_ERR_INVALID_ARG
    m = W.paint_layer(n_wl=8)
    r = gpu_mie(m, allow=(fos.FOS_ERR_INJECTED,), flags=fos.FOS_TEST_INJECT)
    assert r["status"] == fos.FOS_ERR_INJECTED
    r = gpu_mie(m)
    assert r["status"] == fos.FOS_OK
