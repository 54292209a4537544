"""The C-ABI shared library builds, loads without a GPU, and exports every
function that include/*.h declares.  No compute call is made here."""
import ctypes
import glob
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        src = open(h).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        src = re.sub(r"//[^\n]*", "", src)
        for m in re.finditer(r"\b(mcl_[a-z0-9_]+)\s*\(", src):
            names.add(m.group(1))
    return sorted(names)


@pytest.fixture(scope="module")
def built_lib():
    from paper_2406_12202_gb300 import build as B
    return B.build()


def test_header_declares_entry_points():
    names = declared_functions()
    for n in ("mcl_init_map", "mcl_update", "mcl_resample"):
        assert n in names


def test_library_exports_every_declared_symbol(built_lib):
    lib = ctypes.CDLL(built_lib)
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_lists_every_declared_symbol():
    import paper_2406_12202_gb300 as M
    assert sorted(M.EXPORTED) == [n for n in declared_functions() if n in M.EXPORTED]
    assert set(declared_functions()) <= set(M.EXPORTED)


def test_last_error_without_gpu(built_lib):
    lib = ctypes.CDLL(built_lib)
    lib.mcl_last_error.restype = ctypes.c_char_p
    assert lib.mcl_last_error() == b""
