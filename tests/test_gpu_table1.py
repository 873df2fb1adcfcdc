"""The network with the paper's own inputs (section "Photon transport", Table 1): slab
features, the Table 1 range gate, and a short train-and-evaluate run against Monte Carlo."""
import math

import numpy as np
import pytest

from paper_2409_00165_gb300 import fos
from paper_2409_00165_gb300 import surrogate as S
from paper_2409_00165_gb300 import workloads as W

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def test_slab_features_closed_form():
    r = W.table1_slabs(5000, 3)
    sl = S.Slabs(r)
    f = sl.features().cpu().numpy().astype(np.float64)
    want = np.column_stack([r["n"], np.log10(r["mu_s"] + 1e-4), np.log10(r["mu_a"] + 1e-4),
                            r["g"], np.log10(r["d"]), np.log10(r["mu_s"] * r["d"] + 1e-6),
                            np.log10(r["mu_a"] * r["d"] + 1e-6), np.log10(1 - r["g"] + 1e-3),
                            np.log10(r["mu_s"] * (1 - r["g"]) * r["d"] + 1e-6)])
    assert np.allclose(f, want.astype(np.float32), rtol=2e-7, atol=2e-7)
    bad = dict(r, d=np.where(np.arange(5000) == 7, 0.0, r["d"]))
    out = torch.zeros((5000, 9), dtype=torch.float32, device="cuda")
    s2 = S.Slabs(bad)
    st = fos.fos_surrogate_features_slab(s2.n, s2.mu_s, s2.mu_a, s2.g, s2.d, out)
    assert st == fos.FOS_ERR_INVALID_ARG


def test_table1_gate_and_short_training():
    res = S.table1_experiment(train_rows=60000, train_photons=4000, steps=1500,
                              test_rows=2000, test_photons=20000, members=2, threshold=1.0)
    assert res["flagged"] == 0          # every test slab lies inside Table 1
    assert max(res["mae"]) < 0.02, res["mae"]
    # rows outside the box are flagged whatever the spread
    tr = S.Slabs(W.table1_slabs(2000, 1))
    f = tr.features()
    stats = S.table1_stats(f)
    sur = S.Surrogate(1, stats, seed=1)
    out = dict(n=[1.5, 7.5, 1.5, 1.5, 1.5, 1.5, 1.0, 7.0], mu_s=[1.0, 1.0, 25.0, 1.0, 0.5, 0.1, 0.0, 20.0],
               mu_a=[0.1, 0.1, 0.1, 150.0, 0.1, 0.1, 0.0, 100.0],
               g=[0.5, 0.5, 0.5, 0.5, 0.5, 0.5, 0.0, 0.99], d=[50.0, 50.0, 1.0, 50.0, 600.0, 4.0, 5.0, 5.0])
    o = S.Slabs({k: np.asarray(v, float) for k, v in out.items()})
    _, _, needs = sur.predict(o.features(), threshold=1.0)
    assert needs.cpu().numpy().tolist() == [0, 1, 1, 1, 1, 1, 0, 0]
