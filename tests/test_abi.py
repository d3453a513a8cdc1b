"""The C ABI library builds for sm_103a, loads without a GPU and exports every entry point that
include/fmm.h declares (no compute call is made here)."""
import ctypes
import os
import re

from paper_1006_2269_gb300 import build

HEADER = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "include")


def declared_functions():
    names = []
    for f in sorted(os.listdir(HEADER)):
        if not f.endswith(".h"):
            continue
        text = open(os.path.join(HEADER, f)).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        names += re.findall(r"^\s*(?:const\s+)?[A-Za-z_][\w\s\*]*?\b(fmm_\w+)\s*\(", text, flags=re.M)
    return sorted(set(names))


def test_header_declares_the_boundary():
    names = declared_functions()
    for must in ("fmm_build_tree", "fmm_interaction_lists", "fmm_evaluate"):
        assert must in names
    assert len(names) >= 14


def test_library_exports_every_declared_symbol():
    lib = ctypes.CDLL(build.build())
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_names_match_the_abi():
    from paper_1006_2269_gb300 import fmm
    for n in declared_functions():
        assert hasattr(fmm, n), n


def test_binding_fails_loudly_without_library(tmp_path):
    # no CPU fallback: a missing library is an error, not a silent slow path
    import pytest

    from paper_1006_2269_gb300 import fmm
    saved = fmm._lib
    try:
        fmm._lib = None
        with pytest.raises(RuntimeError):
            fmm.load_library(str(tmp_path / "missing.so"))
    finally:
        fmm._lib = saved
