"""The C-ABI library builds for sm_103a, loads, and exports every symbol of include/*.h.

No compute call here: this runs on machines without a GPU.
"""
import ctypes
import glob
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared_functions():
    names = []
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        text = open(h).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        for m in re.finditer(r"^\s*(?:const\s+)?[A-Za-z_][A-Za-z0-9_\s\*]*?\b(fos_[a-z0-9_]+)\s*\(",
                             text, flags=re.M):
            names.append(m.group(1))
    return sorted(set(names))


@pytest.fixture(scope="module")
def libfos():
    from paper_2409_00165_gb300 import build
    path = build.build()
    return ctypes.CDLL(path)


def test_header_declares_the_boundary():
    names = _declared_functions()
    for must in ("fos_mie_properties", "fos_mc_spectrum", "fos_status_string",
                 "fos_sync_status", "fos_mc_autotune"):
        assert must in names


def test_every_declared_symbol_is_exported(libfos):
    missing = [n for n in _declared_functions() if not hasattr(libfos, n)]
    assert not missing, missing


def test_status_strings_and_version(libfos):
    libfos.fos_status_string.restype = ctypes.c_char_p
    libfos.fos_status_string.argtypes = [ctypes.c_int]
    assert libfos.fos_status_string(0) == b"ok"
    assert b"invalid" in libfos.fos_status_string(1)
    assert libfos.fos_api_version() == 1


def test_host_side_validation_needs_no_device(libfos):
    from paper_2409_00165_gb300 import fos
    f = fos.lib()
    # NULL batch and empty shapes are rejected before any CUDA call
    assert f.fos_mc_spectrum(None, None, None, 0, 0, None) == fos.FOS_ERR_INVALID_ARG
    b = fos.FosBatch()
    b.n_stacks, b.n_wl, b.max_layers = 0, 1, 1
    assert f.fos_mc_spectrum(ctypes.byref(b), None, None, 0, 0, None) == fos.FOS_ERR_INVALID_ARG
    b.n_stacks, b.max_layers = 1, fos.FOS_MAX_LAYERS + 1
    assert f.fos_mc_spectrum(ctypes.byref(b), None, None, 0, 0, None) == fos.FOS_ERR_INVALID_ARG
    # a photon count that does not fit the 32-bit photon id is refused on the host
    b.max_layers = 1
    b.mu_s = b.mu_a = b.g = b.n_layer = b.thickness = 8
    b.photons_per_item = 2 ** 32
    c = ctypes.c_longlong(0)
    assert f.fos_mc_spectrum(ctypes.byref(b), ctypes.byref(c), None, 0, 0, None) == \
        fos.FOS_ERR_INVALID_ARG
    assert f.fos_mc_set_tuning(48, 8) == fos.FOS_ERR_INVALID_ARG
    assert f.fos_mc_set_tuning(288, 8) == fos.FOS_ERR_INVALID_ARG   # above the largest variant
    assert f.fos_mc_set_tuning(256, 8) == fos.FOS_OK
    assert f.fos_mc_set_tuning(0, 0) == fos.FOS_OK
    assert f.fos_mie_properties(0, None, 1, None, None, 0, None, None, None, None, None,
                                None, None, None, None, None, None, 0, None) == \
        fos.FOS_ERR_INVALID_ARG


def test_binary_targets_sm_103a():
    from paper_2409_00165_gb300 import build
    assert "arch=compute_103a,code=sm_103a" in " ".join(build.ARCH)
