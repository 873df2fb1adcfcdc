"""The hardware-rate diagnostic runs, returns positive rates, and orders them as the
kernels' designs assume: N = 128 and 256 run the tensor pipe at the same rate, N = 64
below it, and the packed half-precision tanh is not a faster way through the MUFU."""
import pytest

from paper_2409_00165_gb300 import fos

pytestmark = pytest.mark.gpu


def test_hw_rates():
    r = fos.fos_measure_hw_rates()
    assert r["fp64_tflops"] > 0.1
    assert r["tanh_per_s"] > 1e11
    assert 0 < r["tanh_f16x2_per_s"] < 1.5 * r["tanh_per_s"]
    assert r["bulk_tbps"] > 1.0
    for kind in ("mma_ts_tflops", "mma_ss_tflops"):
        t = r[kind]
        assert all(v > 100.0 for v in t.values())
        assert abs(t[128] - t[256]) < 0.1 * t[256]
        assert t[64] < 0.9 * t[128]
