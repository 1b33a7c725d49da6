"""Host-side checks of the C ABI: the library loads without a GPU and exports
every entry point declared in include/kfbi.h; argument errors are reported
without touching a device."""
import ctypes as C
import os
import re

import pytest

from paper_2104_05024_gb300 import kfbi as K

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    src = open(os.path.join(ROOT, "include", "kfbi.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"^\s*(?:const\s+)?\w+\**\s+\**(\w+)\s*\(", src, flags=re.M)))


def _lib():
    try:
        return K.load()
    except OSError as e:
        pytest.skip(f"library not built: {e}")


def test_header_declares_expected_entry_points():
    names = declared_functions()
    for n in ("kfbi_create", "kfbi_solve_neumann", "bidomain_step", "kfbi_destroy"):
        assert n in names


def test_library_exports_every_declared_symbol():
    lib = _lib()
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing
    assert set(K.EXPORTS) <= set(declared_functions())


def test_null_arguments_rejected_without_gpu():
    lib = _lib()
    h = C.c_void_p()
    rc = lib.kfbi_create(None, None, 1.0, 2.0, 0.05, None, C.byref(h))
    assert rc == K.ERR_ARG
    assert b"null" in lib.kfbi_last_error()
    assert lib.kfbi_solve_neumann(None, 1.0, None, None, None, None, None) == K.ERR_ARG
    assert lib.kfbi_react_fe(None, 0.1, None, None, 0, None) == K.ERR_ARG
