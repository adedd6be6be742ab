"""The C ABI library loads and exports every entry point include/hbgls.h declares (no GPU needed)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "hbgls.h")


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    names = re.findall(r"^\s*(?:hb_status|const char \*|int64_t|int)\s*\**\s*(hb_\w+)\s*\(", text, flags=re.M)
    return sorted(set(names))


@pytest.fixture(scope="module")
def libpath():
    from paper_2411_14315_gb300 import build
    return build.build()


def test_header_declares_entry_points():
    names = declared_functions()
    for n in ["hb_create", "hb_destroy", "hb_residual", "hb_jv", "hb_jv_dev", "hb_solve", "hb_get_harmonics"]:
        assert n in names


def test_library_exports_every_declared_symbol(libpath):
    lib = ctypes.CDLL(libpath)
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_covers_every_declared_symbol():
    from paper_2411_14315_gb300 import hbgls
    assert set(declared_functions()) <= set(hbgls.SIGNATURES)


def test_errors_without_device_are_reported_not_raised(libpath):
    """hb_create on a missing device returns a status and a message (no crash, no exception)."""
    from paper_2411_14315_gb300 import hbgls
    lib = hbgls.lib()
    m = hbgls.hb_mesh()
    h = ctypes.c_void_p()
    st = lib.hb_create(ctypes.byref(m), 1.0, 1.0, 1.0, 1, 0, None, ctypes.byref(h))
    assert st != 0
    assert lib.hb_last_error().decode()
