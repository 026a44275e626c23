"""The C-ABI library builds for sm_103a, loads, and exports every function
that include/*.h declares (no compute calls: no GPU needed)."""
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
        for m in re.finditer(r"^\s*(?:const\s+)?[A-Za-z_][A-Za-z0-9_]*\s*\**\s*([a-z][a-z0-9_]*)\s*\(", src, flags=re.M):
            names.add(m.group(1))
    return sorted(names)


@pytest.fixture(scope="module")
def lib():
    from paper_2510_01495_gb300 import _build
    path = _build.build()
    return ctypes.CDLL(path)


def test_header_declares_entry_points():
    names = declared_functions()
    for must in ("ttv_single", "ttv_multi", "ttv_out_free", "ttv_last_error"):
        assert must in names


@pytest.mark.parametrize("name", declared_functions())
def test_symbol_exported(lib, name):
    assert hasattr(lib, name), f"{name} declared in include/ but not exported"


def test_product_has_no_oracle_dependency():
    """The library sources never include or call the oracle."""
    for f in glob.glob(os.path.join(ROOT, "paper_2510_01495_gb300", "**", "*.*"), recursive=True):
        if f.endswith((".cu", ".cuh", ".cpp", ".h", ".py")):
            txt = open(f, errors="replace").read()
            assert "oracle" not in txt.lower().replace("the oracle", ""), f
