"""CPU-side checks of the C ABI: the library builds, loads without a GPU and
exports every function include/dtr.h declares; argument validation that needs
no device works."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "dtr.h")


@pytest.fixture(scope="module")
def lib():
    from paper_1603_05988_gb300 import build
    if not os.path.exists(build.LIB):
        build.build()
    return ctypes.CDLL(build.LIB)


def declared_functions():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    names = re.findall(r"\b(dtr_[a-z0-9_]+)\s*\(", src)
    return sorted(set(names))


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ["dtr_make_lattice", "dtr_make_gauge", "dtr_gauge_from_host", "dtr_dslash", "dtr_gen_noise", "dtr_solve_batch",
                     "dtr_deflate_project", "dtr_trace_estimate", "dtr_defl_create", "dtr_last_error"]:
        assert required in names


def test_library_exports_every_declared_symbol(lib):
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_lattice_validation_without_gpu(lib):
    lib.dtr_make_lattice.restype = ctypes.c_int
    lib.dtr_last_error.restype = ctypes.c_char_p
    h = ctypes.c_void_p()
    dims = (ctypes.c_int * 4)(4, 4, 4, 3)
    assert lib.dtr_make_lattice(dims, ctypes.byref(h)) == 1          # DTR_EINVAL: odd extent
    assert b"even" in lib.dtr_last_error()
    dims = (ctypes.c_int * 4)(4, 4, 4, 8)
    assert lib.dtr_make_lattice(dims, ctypes.byref(h)) == 0
    V = ctypes.c_int64()
    Nd = ctypes.c_int64()
    lib.dtr_lattice_info.restype = ctypes.c_int
    assert lib.dtr_lattice_info(h, None, ctypes.byref(V), ctypes.byref(Nd)) == 0
    assert V.value == 512 and Nd.value == 12 * 512
    lib.dtr_destroy_lattice(h)


def test_binding_mirrors_the_abi():
    from paper_1603_05988_gb300 import build
    if not os.path.exists(build.LIB):
        build.build()
    from paper_1603_05988_gb300 import dtr
    for name in ["make_lattice", "make_gauge", "gauge_from_host", "dslash", "gen_noise", "solve_batch", "defl_create",
                 "deflate_project", "trace_estimate"]:
        assert callable(getattr(dtr, name))
    assert "sm_103a" in dtr.version()
