"""The synthetic inputs follow the recipes stated for them (no GPU): grids, closed-form
materials, seeded design draws and their ranges, the oversampled shares of the training
sets, and determinism under a fixed seed."""
import numpy as np

from paper_2409_00165_gb300 import workloads as W


def test_wavelength_grid_and_paint_materials():
    wl = W.wavelengths(400)
    assert wl.shape == (400,) and wl[0] == 0.3 and wl[-1] == 2.5
    assert np.allclose(np.diff(wl), 2.2 / 399)
    npart = W.particle_index(wl)
    assert np.allclose(npart.real, 2.5 + 0.05 / wl ** 2)
    assert np.all(npart.imag[wl < 0.4] == 0.5) and np.all(npart.imag[wl >= 0.4] == 1e-4)
    nm = W.matrix_index(wl)
    assert np.all(nm.real == 1.48) and np.allclose(nm.imag, 1e-5 * wl)


def test_paint_layer_recipe():
    m = W.paint_layer()
    assert m["n_wl"] == 400 and m["photons_per_item"] == 1000000 and m["seed"] == 1
    assert np.all(m["radius"] == 0.2) and np.all(m["vol_frac"] == 0.10)
    assert np.all(m["thickness"] == 300.0) and m["substrate_R"] is None
    assert m["n_p"].shape == (1, 400) and m["nm"].shape == (1, 400)


def test_layer_stack_batch_recipe():
    a, b = W.layer_stacks(), W.layer_stacks()
    assert np.array_equal(a["radius"], b["radius"]) and np.array_equal(a["n_photons"],
                                                                       b["n_photons"])
    assert a["n_stacks"] == 64 and a["n_wl"] == 200 and a["max_layers"] == 3
    assert set(np.unique(a["n_layers"])) <= {1, 2, 3}
    assert len(a["species_group"]) == a["n_layers"].sum()
    assert np.all((a["radius"] >= 0.05) & (a["radius"] <= 1.0))
    assert np.all((a["vol_frac"] >= 0.01) & (a["vol_frac"] <= 0.3))
    assert np.all((a["thickness"] >= 10.0) & (a["thickness"] <= 500.0))
    n = a["n_photons"]
    assert n.shape == (64 * 200,) and n.min() >= 10000 and n.max() <= 1000000
    assert np.all(a["substrate_R"] == 0.05)
    # budgets log-uniform: about half of them below the geometric middle 1e5
    assert 0.4 < np.mean(n < 100000) < 0.6


def test_single_layer_designs_and_log_share():
    u = W.single_layer_designs(200000, seed=4)
    assert np.all((u["radius"] >= 0.05) & (u["radius"] <= 1.0))
    assert np.all((u["vol_frac"] >= 0.01) & (u["vol_frac"] <= 0.3))
    assert np.all((u["thickness"] >= 10.0) & (u["thickness"] <= 500.0))
    assert np.allclose(u["wl"], W.wavelengths(300))
    h = W.single_layer_designs(200000, seed=4, log_share=0.5)
    assert np.all((h["vol_frac"] >= 0.01) & (h["vol_frac"] <= 0.3))
    # uniform f puts 1/29 of the designs below f = 0.02; half log-uniform adds
    # 0.5 * ln 2 / ln 30 of them
    low_u, low_h = np.mean(u["vol_frac"] < 0.02), np.mean(h["vol_frac"] < 0.02)
    assert abs(low_u - 0.01 / 0.29) < 0.003
    assert abs(low_h - (0.5 * 0.01 / 0.29 + 0.5 * np.log(2) / np.log(30))) < 0.005
    r = W.single_layer_designs(1000, seed=9, random_wl=True)
    assert r["wl"].shape == (1000,) and np.all((r["wl"] >= 0.3) & (r["wl"] <= 2.5))


def test_table1_slabs_stay_in_the_table_box():
    s = W.table1_slabs(200000, seed=40, g_log_share=0.5, n_log_share=0.3)
    t = W.TABLE1
    assert np.all((s["n"] >= t["n"][0]) & (s["n"] <= t["n"][1]))
    assert np.all((s["g"] >= t["g"][0]) & (s["g"] <= t["g"][1]))
    assert np.all((s["d"] >= t["d"][0]) & (s["d"] <= t["d"][1]))
    assert np.all((s["mu_s"] >= 0) & (s["mu_s"] <= t["mu_s"][1] * (1 + 1e-12)))
    assert np.all((s["mu_a"] >= 0) & (s["mu_a"] <= t["mu_a"][1] * (1 + 1e-12)))
    assert np.all(s["mu_s"] * s["d"] <= t["tau_s_max"] * (1 + 1e-12))
    assert abs(np.mean(s["mu_s"] == 0) - 0.05) < 0.005
    assert abs(np.mean(s["mu_a"] == 0) - 0.05) < 0.005
    # oversampled corners: g near 1 and n near 1
    plain = W.table1_slabs(200000, seed=40)
    assert np.mean(s["g"] > 0.95) > 2 * np.mean(plain["g"] > 0.95)
    assert np.mean(s["n"] < 1.05) > 5 * np.mean(plain["n"] < 1.05)


def test_size_distribution_and_core_shell_materials():
    wl = W.wavelengths(50)
    si = W.silicon_like_index(wl)
    assert np.allclose(si, (3.45 + 0.2 / wl ** 2) + 1j * 0.5 * np.exp(-(wl - 0.3) / 0.1))
    h2o = W.water_like_index(wl)
    assert np.allclose(h2o, 1.33 + 1j * (1e-7 + 1e-5 * wl ** 4))
    sio2 = W.silica_like_index(wl)
    assert np.all((sio2.real > 1.4) & (sio2.real < 1.5)) and np.all(sio2.imag > 0)
    m = W.hollow_silica_media()
    assert np.allclose(m["radius"], [0.35, 0.45, 0.55, 0.35, 0.45, 0.55])
    assert np.allclose(m["core_radius"], [0.25, 0.25, 0.25, 0, 0, 0])
    assert np.all(m["vol_frac"] == 0.6) and np.all(m["thickness"] == 50.0)
    assert np.all(m["nm"] == 1.0) and np.all(m["n_core"] == 1.0)


def test_conductor_and_solar_stand_ins():
    wl = W.wavelengths(400)
    al = W.aluminium_like_index(wl)
    eps = 1.0 - (wl / 0.083) ** 2 / (1.0 + 1j * wl / 12.4)
    assert np.allclose(al * al, eps) and np.all(al.imag > 0)
    # a good conductor over the grid: reflectance at normal incidence from air > 0.85
    r = np.abs((1 - al) / (1 + al)) ** 2
    assert np.all(r > 0.85)
    g = W.solar_like_irradiance(wl)
    assert np.all(g > 0) and abs(g[np.argmin(np.abs(wl - 0.5))] - 1.0) < 0.01
    # Wien's law: the 5778 K peak sits near 0.50 um
    fine = np.linspace(0.3, 1.0, 7001)
    assert abs(fine[np.argmax(W.solar_like_irradiance(fine))] - 2897.77 / 5778.0) < 1e-3
    m = W.oblique_conductor_media()
    assert np.allclose(m["cos_incidence"][::400], [1.0, np.cos(np.pi / 6), 0.5])
    assert np.allclose(m["n_below"][:400], al.real) and np.allclose(m["k_below"][:400], al.imag)
