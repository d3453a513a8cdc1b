"""Argument checks of the C ABI that happen on the host, before any device work (CPU only)."""
import ctypes

import pytest

from paper_1006_2269_gb300 import build, fmm


@pytest.fixture(scope="module")
def lib():
    build.build()
    return fmm.load_library()


def test_levels_check(lib):
    h = ctypes.c_void_p()
    assert lib.fmm_tree_create(15, 2, ctypes.byref(h)) == fmm.FMM_ERR_LEVELS
    assert b"4^2" in lib.fmm_last_error()
    assert lib.fmm_tree_create(100, -1, ctypes.byref(h)) == fmm.FMM_ERR_ARG
    assert lib.fmm_tree_create(100, 14, ctypes.byref(h)) == fmm.FMM_ERR_ARG
    assert lib.fmm_tree_create(0, 0, ctypes.byref(h)) == fmm.FMM_ERR_ARG
    assert lib.fmm_tree_create(1 << 31, 1, ctypes.byref(h)) == fmm.FMM_ERR_ARG
    assert not h.value


def test_null_handles(lib):
    assert lib.fmm_build_tree(None, None, None, None) == fmm.FMM_ERR_ARG
    assert lib.fmm_interaction_lists(None, None, 0.5, None) == fmm.FMM_ERR_ARG
    assert lib.fmm_evaluate(None, None, None, None, None, None) == fmm.FMM_ERR_ARG
    assert lib.fmm_lists_sync(None, None, None, None) == fmm.FMM_ERR_ARG
    assert lib.fmm_direct(None, None, None, 10, None, 1, None, None) == fmm.FMM_ERR_ARG
    lib.fmm_tree_destroy(None)
    lib.fmm_lists_destroy(None)
