"""fos_mc_spectrum_noalloc: the photon walk for callers that cannot allocate device memory.

Callers whose device memory is all owned by another allocator, or that run under a
fixed memory budget, cannot call cudaMalloc.  For them the library offers an entry
point whose scratch is a fixed static device array.  These tests call it through the
C-ABI and check that it returns exactly the counts of fos_mc_spectrum on the same
batch, on two calls in a row (the array keeps the previous call's contents, so the
second call shows the state is cleared), and that an over-size batch is refused.

This file sorts last so that a run stopping at its first failure has already run
every other test.
"""
import numpy as np
import pytest

from gpu_helpers import to_dev
from paper_2409_00165_gb300 import fos

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def _batch(n_st, L, seed, photons):
    rng = np.random.default_rng(seed)
    f64 = torch.float64
    t = dict(n_layers=to_dev(rng.integers(1, L + 1, size=n_st).astype(np.int32), torch.int32),
             mu_s=to_dev(rng.uniform(0, 20, size=n_st * L), f64),
             mu_a=to_dev(rng.uniform(0, 2, size=n_st * L), f64),
             g=to_dev(rng.uniform(-0.5, 0.95, size=n_st * L), f64),
             n_layer=to_dev(rng.uniform(1.0, 2.0, size=n_st * L), f64),
             thickness=to_dev(rng.uniform(0.05, 0.5, size=n_st * L), f64),
             n_above=to_dev(rng.uniform(1.0, 1.4, size=n_st), f64),
             n_below=to_dev(rng.uniform(1.0, 1.6, size=n_st), f64),
             n_photons=to_dev(rng.integers(0, photons, size=n_st).astype(np.int64), torch.int64))
    b = fos.make_batch(n_st, 1, L, seed=seed, **t)
    return b, t


def _counts(n):
    return torch.full((n, fos.FOS_NCOUNT), -7, dtype=torch.int64, device="cuda")


def test_noalloc_matches_fos_mc_spectrum_twice():
    b, keep = _batch(53, 3, 2024, 5000)
    ref = _counts(53)
    fos.check(fos.fos_mc_spectrum(b, ref, None, 0, 0), "fos_mc_spectrum")
    for _ in range(2):
        out = _counts(53)
        fos.check(fos.fos_mc_spectrum_noalloc(b, out), "fos_mc_spectrum_noalloc")
        torch.cuda.synchronize()
        assert torch.equal(out, ref)
    # a different, larger batch right after: nothing left over from the previous call
    b2, keep2 = _batch(700, 2, 7, 3000)
    ref2 = _counts(700)
    fos.check(fos.fos_mc_spectrum(b2, ref2, None, 0, 0), "fos_mc_spectrum")
    out2 = _counts(700)
    fos.check(fos.fos_mc_spectrum_noalloc(b2, out2), "fos_mc_spectrum_noalloc")
    assert torch.equal(out2, ref2)
    assert torch.equal(out2[:, :4].sum(dim=1), keep2["n_photons"])


def test_noalloc_refuses_batches_beyond_its_maximum():
    n = fos.FOS_NOALLOC_MAX_ITEMS + 1
    f64 = torch.float64
    ones = torch.ones(n, dtype=f64, device="cuda")
    b = fos.make_batch(n, 1, 1, ones * 2.0, ones * 0.1, ones * 0.5, ones * 1.5, ones,
                       photons_per_item=10, seed=1)
    out = _counts(n)
    st = fos.fos_mc_spectrum_noalloc(b, out)
    assert st == fos.FOS_ERR_OUT_OF_RANGE
    assert torch.all(out == -7)   # no device work was done
    assert fos.fos_mc_spectrum_noalloc(b, out, flags=fos.FOS_ASYNC) == fos.FOS_ERR_INVALID_ARG


_FILLED = r"""
import sys
import torch
sys.path[:0] = [{root!r}, {tests!r}]
from paper_2409_00165_gb300 import fos
from test_zz_no_alloc import _batch, _counts
torch.cuda.set_device(0)
b, keep = _batch(300, 3, 99, 4000)
ref = _counts(300)
fos.check(fos.fos_mc_spectrum(b, ref, None, 0, 0), "fos_mc_spectrum")
ref = ref.cpu()
outs = [_counts(300) for _ in range(3)]
fos.check(fos.fos_mc_spectrum_noalloc(b, outs[0]), "first call")   # the per-device set-up
torch.cuda.synchronize()
assert torch.equal(outs[0].cpu(), ref)
# take every block of device memory that can still be had
held = []
chunk = 8 << 30
while chunk >= (1 << 20):
    try:
        held.append(torch.empty(chunk, dtype=torch.uint8, device="cuda"))
    except torch.cuda.OutOfMemoryError:
        chunk //= 2
free, total = torch.cuda.mem_get_info()
print("device memory free after the fill (MiB):", free >> 20, "of", total >> 20, flush=True)
for k in (1, 2):
    fos.check(fos.fos_mc_spectrum_noalloc(b, outs[k]), f"call {{k}} with the device full")
    torch.cuda.synchronize()
    assert torch.equal(outs[k].cpu(), ref), k
print("ok", flush=True)
"""


def test_noalloc_runs_with_device_memory_full():
    """After its first call on a device, the entry point needs no device memory at all:
    in a fresh process, one call, then all the device memory that can still be had taken
    by another allocator (torch), then two more calls that still return
    fos_mc_spectrum's counts."""
    import os
    import subprocess
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    tests = os.path.join(root, "tests")
    code = _FILLED.format(root=root, tests=tests)
    r = subprocess.run([sys.executable, "-c", code], cwd=root, capture_output=True, text=True,
                       timeout=600)
    assert r.returncode == 0 and "ok" in r.stdout, (r.stdout[-2000:], r.stderr[-4000:])
