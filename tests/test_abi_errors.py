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


def test_noalloc_short_outputs_refused_before_launch(lib):
    # fmm_build_tree_noalloc writes 4 * nbox doubles into rects and 4^L + 1 ints into leaf_begin
    # through raw pointers: the binding refuses shorter buffers before the library is called
    import torch
    n, L = 1000, 3
    nbox = (4 ** (L + 1) - 1) // 3
    x = torch.zeros(n, dtype=torch.float64)
    perm = torch.empty(n, dtype=torch.int32)
    lb = torch.empty(4 ** L + 1, dtype=torch.int32)
    with pytest.raises(fmm.FMMError, match="rects has 336 elements, needs 340"):
        fmm.fmm_build_tree_noalloc(x, x, L, perm, torch.empty((nbox - 1, 4), dtype=torch.float64), lb)
    with pytest.raises(fmm.FMMError, match="leaf_begin has 64 elements, needs 65"):
        fmm.fmm_build_tree_noalloc(x, x, L, perm, torch.empty((nbox, 4), dtype=torch.float64),
                                   torch.empty(4 ** L, dtype=torch.int32))
    with pytest.raises(fmm.FMMError, match="perm has 999 elements"):
        fmm.fmm_build_tree_noalloc(x, x, L, torch.empty(n - 1, dtype=torch.int32),
                                   torch.empty((nbox, 4), dtype=torch.float64), lb)


def test_shape_setters_check_their_handle(lib):
    assert lib.fmm_set_near_shape(None, 2) == fmm.FMM_ERR_ARG
    assert lib.fmm_get_near_shape(None, None) == fmm.FMM_ERR_ARG
    assert lib.fmm_set_m2l_shape(None, 16, 1) == fmm.FMM_ERR_ARG
