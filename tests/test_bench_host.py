"""Host-side parts of bench.py that need no GPU: the summary of the SM-clock samples taken
during the timed region (median clock, maximum, throttle reasons seen)."""
import importlib.util
import os
import tempfile

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _bench():
    spec = importlib.util.spec_from_file_location("bench_mod", os.path.join(ROOT, "bench.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


def test_clock_summary_reads_samples_and_reasons():
    b = _bench()
    s = b.ClockSampler(0)
    fd, s.path = tempfile.mkstemp(suffix=".csv")
    with os.fdopen(fd, "w") as f:
        f.write("0, 2070, 2070, 900.1, 0x0, Not Active, Not Active, Not Active, Not Active\n")
        f.write("0, 1980, 2070, 1390.5, 0x4, Not Active, Not Active, Not Active, Active\n")
        f.write("0, 2070, 2070, 1000.0, 0x0, Not Active, Not Active, Not Active, Not Active\n")
        f.write("garbage line\n")
        f.write("0, [N/A], 2070, 1.0, 0x0, Not Active, Not Active, Not Active, Not Active\n")
    r = s.summary()
    assert r == dict(sm_mhz=2070.0, sm_max_mhz=2070.0, reasons=["sw_power_cap"], samples=3)
    assert not os.path.exists(s.path)


def test_clock_summary_flags_thermal_slowdown():
    b = _bench()
    s = b.ClockSampler(0)
    fd, s.path = tempfile.mkstemp(suffix=".csv")
    with os.fdopen(fd, "w") as f:
        f.write("0, 1500, 2070, 1400, 0x20, Not Active, Not Active, Active, Not Active\n")
        f.write("0, 1400, 2070, 1400, 0x48, Active, Active, Not Active, Not Active\n")
    r = s.summary()
    assert r["sm_mhz"] == 1450.0 and r["samples"] == 2
    assert r["reasons"] == ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown"]


def test_clock_summary_without_samples():
    b = _bench()
    s = b.ClockSampler(0)
    assert s.summary() is None
