"""Host-only checks of the C ABI: the library builds for sm_103a, loads, and exports every entry
point that include/xflat.h declares (no compute calls: this runs without a GPU)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "xflat.h")


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(?:int|const char\*)\s+(xflat_\w+)\s*\(", text)))


@pytest.fixture(scope="module")
def lib_path():
    from paper_1912_10596_gb300 import build
    return build.build()


def test_header_declares_the_boundary():
    names = declared_functions()
    for core in ("xflat_create", "xflat_set_spectra", "xflat_evolve", "xflat_moments",
                 "xflat_get_rho", "xflat_destroy", "xflat_adjoint", "xflat_evolve_batch"):
        assert core in names


def test_library_exports_every_declared_symbol(lib_path):
    lib = ctypes.CDLL(lib_path)
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_status_strings_and_defaults_without_gpu(lib_path):
    lib = ctypes.CDLL(lib_path)
    lib.xflat_status_string.restype = ctypes.c_char_p
    assert lib.xflat_status_string(0) == b"ok"
    assert lib.xflat_status_string(4) == b"device barrier timeout"
    from paper_1912_10596_gb300 import xflat
    c = xflat.default_config()
    assert c.abi_version == xflat.ABI_VERSION == 2 and c.n_flavor == 2 and c.R_km == 11.0
    assert c.geometry == xflat.GEOMETRY_BULB and c.mu_const_kmi == 0.0
    assert ctypes.sizeof(xflat.xflat_config) == 224


def test_create_rejects_bad_config_before_touching_the_gpu(lib_path):
    from paper_1912_10596_gb300 import xflat
    c = xflat.default_config()
    c.n_flavor = 4
    h = ctypes.c_void_p()
    assert xflat.xflat_create(ctypes.byref(c), ctypes.byref(h)) == xflat.ERR_INVAL
    c = xflat.default_config()
    c.abi_version = 99
    assert xflat.xflat_create(ctypes.byref(c), ctypes.byref(h)) == xflat.ERR_INVAL
    c = xflat.default_config()
    c.integrator = xflat.LIE_ADAPTIVE
    c.n_flavor = 3
    c.n_phi = 4                                     # the extended model is two-flavour only
    assert xflat.xflat_create(ctypes.byref(c), ctypes.byref(h)) == xflat.ERR_UNSUPPORTED
    c = xflat.default_config()
    c.integrator = xflat.LIE_ADAPTIVE
    c.n_phi = 4
    assert xflat.xflat_create(ctypes.byref(c), ctypes.byref(h)) == xflat.ERR_UNSUPPORTED
    c = xflat.default_config()
    c.integrator = 5
    assert xflat.xflat_create(ctypes.byref(c), ctypes.byref(h)) == xflat.ERR_INVAL
    c = xflat.default_config()
    c.geometry = 3
    assert xflat.xflat_create(ctypes.byref(c), ctypes.byref(h)) == xflat.ERR_INVAL
    c = xflat.default_config()
    c.geometry = xflat.GEOMETRY_SINGLE_ANGLE
    c.n_phi = 4
    assert xflat.xflat_create(ctypes.byref(c), ctypes.byref(h)) == xflat.ERR_UNSUPPORTED
    c = xflat.default_config()
    c.matter_kind = 4
    assert xflat.xflat_create(ctypes.byref(c), ctypes.byref(h)) == xflat.ERR_INVAL
