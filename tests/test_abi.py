"""The C-ABI library builds for sm_103a, loads without a GPU and exports every
function that include/cjt.h declares (no compute calls here)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_1602_02618_gb300 import build
    path = build.build()
    return ctypes.CDLL(path)


def declared_functions():
    text = open(os.path.join(ROOT, "include", "cjt.h")).read()
    text = re.sub(r"/\*.*?\*/", " ", text, flags=re.S)
    return sorted(set(re.findall(r"\b(cjt_\w+)\s*\(", text)))


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ("cjt_plan", "cjt_forward", "cjt_inverse", "cjt_execute_batched", "cjt_destroy",
                     "cjt_strerror", "cjt_sync", "cjt_execute_host"):
        assert required in names


def test_library_exports_every_declared_symbol(lib):
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_host_only_calls(lib):
    lib.cjt_strerror.restype = ctypes.c_char_p
    assert lib.cjt_strerror(0) == b"success"
    assert b"alpha" in lib.cjt_strerror(-2)
    lib.cjt_version.restype = ctypes.c_char_p
    assert b"sm_103a" in lib.cjt_version()


def test_binding_names_match_header():
    from paper_1602_02618_gb300 import cjt
    assert sorted(cjt.EXPORTED) == declared_functions()
