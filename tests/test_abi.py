"""The C-ABI library builds, loads and exports every entry point that
include/mpw.h declares (no GPU needed: nothing here launches a kernel)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    src = open(os.path.join(ROOT, "include", "mpw.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    names = re.findall(r"^[A-Za-z_][\w \*]*?\b(mpw_\w+)\s*\(", src, flags=re.M)
    return sorted(set(names))


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ("mpw_create", "mpw_create_patch", "mpw_set_fields", "mpw_step", "mpw_get_fields",
                     "mpw_destroy"):
        assert required in names


def test_library_exports_every_declared_symbol(mpw_lib):
    lib = ctypes.CDLL(mpw_lib.LIB_PATH)
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing
    # the Python binding covers the same set, nothing more
    assert sorted(mpw_lib.SIGNATURES) == declared_functions()


def test_binding_refuses_to_run_without_the_library(mpw_lib, tmp_path, monkeypatch):
    """No CPU fallback: a missing libmpw.so is an import error."""
    monkeypatch.setattr(mpw_lib, "LIB_PATH", str(tmp_path / "missing.so"))
    with pytest.raises(ImportError):
        mpw_lib._load()
