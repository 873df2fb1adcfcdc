"""Pins of the oracle's random-number and FP32 series functions."""
import os

import numpy as np
import pytest

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _kat():
    rows = []
    with open(os.path.join(GOLDEN, "philox4x32_10_kat.txt")) as fh:
        for line in fh:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            w = [int(t, 16) for t in line.split()]
            rows.append((w[0:4], w[4:6], w[6:10]))
    return rows


def test_philox_known_answers(orc):
    rows = _kat()
    assert len(rows) == 3
    for ctr, key, want in rows:
        got = orc.philox4x32_10(ctr, key)
        assert [int(v) for v in got] == want


def test_philox_counter_sensitivity(orc):
    # Each counter word and key word changes the output (all 4 words differ).
    base = orc.philox4x32_10([1, 2, 3, 4], [5, 6])
    for i in range(4):
        c = [1, 2, 3, 4]
        c[i] ^= 1
        assert np.all(orc.philox4x32_10(c, [5, 6]) != base)
    for i in range(2):
        k = [5, 6]
        k[i] ^= 1
        assert np.all(orc.philox4x32_10([1, 2, 3, 4], k) != base)


def test_uniform_open_interval_and_exact(orc):
    assert orc.uniform(0) == 2.0 ** -24
    assert orc.uniform(0xFFFFFFFF) == 1.0 - 2.0 ** -24
    assert orc.uniform(1 << 9) == 3 * 2.0 ** -24
    # the 9 low bits are dropped
    assert orc.uniform(0x1FF) == orc.uniform(0)
    vals = [orc.uniform(x) for x in (0x12345678, 0x9ABCDEF0, 0x80000000)]
    for v in vals:
        assert np.float64(np.float32(v)) == v  # exact in float


def _all_uniforms():
    k = np.arange(2 ** 23, dtype=np.uint64)
    return ((2 * k + 1).astype(np.float64) * 2.0 ** -24).astype(np.float32)


def test_neg_log_f32_exhaustive(orc):
    """-ln(u) of the FP32 mirror is within 2 ulp of libm over every possible u."""
    u = _all_uniforms()
    got = orc.neg_log_f32(u).astype(np.float64)
    ref = -np.log(u.astype(np.float64))
    ulp = np.spacing(np.abs(ref).astype(np.float32)).astype(np.float64)
    assert np.max(np.abs(got - ref) / ulp) <= 2.0
    assert np.all(got > 0)


def test_cos2pi_f32_exhaustive(orc):
    """cos(2 pi u) of the FP32 mirror is within 2^-23 of libm over every possible u."""
    u = _all_uniforms()
    got = orc.cos2pi_f32(u).astype(np.float64)
    ref = np.cos(2.0 * np.pi * u.astype(np.float64))
    assert np.max(np.abs(got - ref)) <= 2.0 ** -23
    assert np.all(np.abs(got) <= 1.0)
    # symmetry cos(2 pi u) = cos(2 pi (1-u)) holds bit for bit (exact reduction)
    assert np.array_equal(got, got[::-1])


def test_philox_uniform_statistics(orc):
    # 4e4 words from consecutive counters: mean and a 16-bin chi-square.
    words = []
    for i in range(10000):
        words.extend(orc.philox4x32_10([i, 7, 0, 0], [1, 0]))
    u = np.array([orc.uniform(int(w)) for w in words])
    n = u.size
    assert abs(u.mean() - 0.5) < 4 * np.sqrt(1 / 12 / n)
    h, _ = np.histogram(u, bins=16, range=(0, 1))
    e = n / 16
    chi2 = np.sum((h - e) ** 2 / e)
    assert chi2 < 40.0  # 15 dof, p ~ 5e-4
