"""The C-ABI library builds for sm_103a, loads without a GPU, and exports every
function that include/vegas.h declares (no compute calls here)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "vegas.h")


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    names = re.findall(r"\b(?:int|void|const char\*)\s+(vegas_\w+)\s*\(", text)
    return sorted(set(names))


@pytest.fixture(scope="module")
def libpath():
    from paper_1503_06182_gb300 import build

    return build.build()


def test_header_declares_the_boundary():
    names = declared_functions()
    for must in ("vegas_init", "vegas_iterate", "vegas_grid_get", "vegas_grid_set", "vegas_adjoint",
                 "vegas_batch_create", "vegas_batch_iterate", "vegas_free", "vegas_strerror"):
        assert must in names


def test_library_exports_every_declared_symbol(libpath):
    lib = ctypes.CDLL(libpath)
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_strerror_without_gpu(libpath):
    lib = ctypes.CDLL(libpath)
    lib.vegas_strerror.restype = ctypes.c_char_p
    assert b"grid" in lib.vegas_strerror(-4)
    assert lib.vegas_strerror(0) == b"ok"


def test_binding_names_match_header():
    from paper_1503_06182_gb300 import vegas

    for n in declared_functions():
        if n in ("vegas_strerror", "vegas_state_size"):
            continue
        assert hasattr(vegas, n), n
