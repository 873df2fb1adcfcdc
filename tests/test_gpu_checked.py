"""The checked build (FOS_CHECKED=1: in-kernel index checks in the walk that set a status
word instead of reading or writing out of bounds, the stand-in for a memory checker):
on ragged multi-item batches under several launch shapes, with photon logs, item lists,
reflectors, conductors and oblique beams, and with the fast walk, no check fires and
the counts and logs equal the oracle's FP32 mirror bit for bit (exact walk)."""
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu

_SCRIPT = r"""
import sys
sys.path[:0] = [{root!r}, {tests!r}]
import numpy as np
import oracle
from gpu_helpers import gpu_mc
from paper_2409_00165_gb300 import fos
from paper_2409_00165_gb300 import build as B
assert fos.lib_path() == B.LIB_CHECKED
rng = np.random.default_rng(17)
n_st, L = 41, 3
b = dict(n_stacks=n_st, n_wl=1, max_layers=L,
         n_layers=rng.integers(1, L + 1, size=n_st).astype(np.int32),
         mu_s=rng.uniform(0, 20, size=n_st * L), mu_a=rng.uniform(0, 2, size=n_st * L),
         g=rng.uniform(-0.5, 0.95, size=n_st * L), n_layer=rng.uniform(1.0, 2.0, size=n_st * L),
         thickness=rng.uniform(0.05, 0.5, size=n_st * L),
         n_above=rng.uniform(1.0, 1.4, size=n_st), n_below=rng.uniform(1.0, 1.6, size=n_st),
         cos_incidence=rng.uniform(0.2, 1.0, size=n_st),
         k_below=np.where(rng.random(n_st) < 0.3, rng.uniform(0.5, 7.0, size=n_st), 0.0),
         n_photons=rng.integers(0, 3000, size=n_st).astype(np.int64), seed=99)
want, want_log = oracle.mc_run(b, fp32=True, photon_log=True)
for tuning in [(0, 0), (64, 1), (256, 16), (96, 3)]:
    fos.fos_mc_set_tuning(*tuning)
    c, log, st = gpu_mc(b, photon_log=True)
    assert st == fos.FOS_OK, (tuning, st)
    assert np.array_equal(c, want) and np.array_equal(log, want_log), tuning
    c, st = gpu_mc(b, flags=fos.FOS_FAST_WALK)
    assert st == fos.FOS_OK and np.array_equal(c[:, :4].sum(axis=1), b["n_photons"]), tuning
fos.fos_mc_set_tuning(0, 0)
b2 = dict(b, item_list=np.array([40, 0, 7, 7, 13], np.int32))
b2.pop("k_below"); b2["substrate_R"] = rng.uniform(0, 1, size=n_st)
want2 = oracle.mc_run(b2, fp32=True)
c2, st = gpu_mc(b2)
assert st == fos.FOS_OK and np.array_equal(c2, want2)
print("ok")
"""


def test_checked_build_fires_no_check_and_matches_the_oracle():
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    code = _SCRIPT.format(root=root, tests=os.path.join(root, "tests"))
    env = dict(os.environ, FOS_CHECKED="1")
    r = subprocess.run([sys.executable, "-c", code], cwd=root, env=env, capture_output=True,
                       text=True, timeout=900)
    assert r.returncode == 0 and "ok" in r.stdout, (r.stdout[-2000:], r.stderr[-4000:])
