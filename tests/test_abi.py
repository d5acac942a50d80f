"""The C-ABI boundary: libgrpic.so builds for sm_103a, loads on a machine
without a GPU and exports every function include/grpic.h declares (no compute
calls here)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared(header):
    text = open(os.path.join(ROOT, "include", header)).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(grpic_[a-z0-9_]+)\s*\(", text)))


@pytest.fixture(scope="module")
def lib():
    from paper_2503_04558_gb300 import build
    path = build.build()
    return ctypes.CDLL(path)


def test_header_declares_the_boundary_calls():
    names = declared("grpic.h")
    for n in ["grpic_init", "grpic_push", "grpic_deposit", "grpic_field_update", "grpic_sort", "grpic_step"]:
        assert n in names


def test_every_declared_symbol_is_exported(lib):
    for hdr in sorted(os.listdir(os.path.join(ROOT, "include"))):
        if hdr.endswith(".h"):
            for name in declared(hdr):
                assert hasattr(lib, name), f"{name} declared in {hdr} but not exported"


def test_binding_lists_match_header():
    from paper_2503_04558_gb300 import grpic as G
    assert sorted(G.EXPORTS) == declared("grpic.h")


def test_binding_refuses_missing_library(tmp_path):
    from paper_2503_04558_gb300 import grpic as G
    with pytest.raises(RuntimeError):
        G.load(str(tmp_path / "nope.so"))
