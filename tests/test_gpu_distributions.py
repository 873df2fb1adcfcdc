"""GPU parity of particle-size distributions (101 sizes per particle) with the oracle."""
import numpy as np
import pytest

from gpu_helpers import gpu_mc, gpu_mie, mc_batch_from_media
from paper_2409_00165_gb300 import fos
from paper_2409_00165_gb300 import workloads as W

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def test_size_distribution_media_parity(orc):
    dists = [fos.fos_size_distribution(0.5, s, 0.001) for s in (0.0, 0.05, 0.15)]
    m = W.size_distribution_media(dists)
    assert len(m["radius"]) == 1 + 101 + 101
    g = gpu_mie(m)
    o = orc.mie_properties(m["wl"], m["nm"], m["species_group"], m["n_p"], m["radius"],
                           m["vol_frac"], n_groups=m["n_groups"])
    for k in ("mu_s", "mu_a", "g"):
        assert np.all(np.abs(g[k] - o[k]) <= 1e-10 * np.abs(o[k])), k
    # the walk on these media agrees with the oracle photon for photon
    b = mc_batch_from_media(m, o, photons=4000)   # the oracle's own coefficients
    b["item_list"] = np.array([0, 57, 199, 400, 777, 1001, 1199], np.int32)
    b["n_above"] = np.ones(m["n_stacks"] * m["n_wl"])
    b["n_below"] = np.ones(m["n_stacks"] * m["n_wl"])
    c_gpu, _ = gpu_mc(b)
    assert np.array_equal(c_gpu, orc.mc_run(b, fp32=True))
    # a distribution smooths the Mie resonances: the spectrum varies less from
    # wavelength to wavelength than the single size's
    rough = [np.abs(np.diff(g["mu_s"][k])).sum() for k in range(3)]
    assert rough[0] > rough[1] > rough[2]
