"""Thin ctypes binding of libfmm_gb300.so (C ABI in include/fmm.h).

Every function has the name of the C entry point it wraps and only marshals arguments: torch
CUDA tensors become device pointers, the current torch stream becomes the cudaStream_t, and a
negative status becomes :class:`FMMError`.  All arithmetic runs in the library's kernels; if the
library is missing this module raises instead of computing anything on the CPU.

:class:`FMM` bundles a tree, its lists and the evaluation for convenience.
"""
from __future__ import annotations

import ctypes
import os
import threading

import torch

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libfmm_gb300.so")
HEADER = os.path.join(os.path.dirname(_HERE), "include", "fmm.h")

FMM_OK = 0
FMM_ERR_ARG = -1
FMM_ERR_NONFINITE = -2
FMM_ERR_LEVELS = -3
FMM_ERR_OOM = -4
FMM_ERR_CUDA = -5
FMM_ERR_CAPACITY = -6
FMM_ERR_TIMEOUT = -7
FMM_ERR_STATE = -8
FMM_ERR_DEGENERATE = -9

FMM_MODE_FP64 = 0
FMM_MODE_MIXED = 1
FMM_MODE_SPLIT = 2


class FMMError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"[{code}] {msg}")
        self.code = code


class fmm_params(ctypes.Structure):
    _fields_ = [("p", ctypes.c_int), ("mode", ctypes.c_int), ("tol", ctypes.c_double)]


_lock = threading.Lock()
_lib = None


def load_library(path: str = LIB_PATH):
    """Load (once) and return the ctypes handle of libfmm_gb300.so."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        if not os.path.exists(path):
            raise RuntimeError(f"{path} is missing: build it with `python -m paper_1006_2269_gb300.build`"
                               " (there is no CPU fallback)")
        lib = ctypes.CDLL(path)
        vp, i64, i32, dbl = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int, ctypes.c_double
        sig = {
            "fmm_tree_create": (i32, [i64, i32, ctypes.POINTER(vp)]),
            "fmm_tree_create_batched": (i32, [i32, vp, vp, ctypes.POINTER(vp)]),
            "fmm_tree_num_instances": (i32, [vp]),
            "fmm_tree_instance": (i32, [vp, i32, ctypes.POINTER(i64), ctypes.POINTER(i64), ctypes.POINTER(i32),
                                        ctypes.POINTER(i64), ctypes.POINTER(i64), ctypes.POINTER(i64)]),
            "fmm_lists_create_batched": (i32, [vp, vp, vp, ctypes.POINTER(vp)]),
            "fmm_lists_counts": (i32, [vp, vp, vp, vp]),
            "fmm_lists_export_instance": (i32, [vp, i32, vp, vp, vp, vp, vp]),
            "fmm_autotune": (i32, [vp, vp, vp, ctypes.POINTER(fmm_params), vp, vp, ctypes.POINTER(i32),
                                   ctypes.POINTER(i32)]),
            "fmm_set_launch": (i32, [vp, i32, i32]),
            "fmm_set_m2l_kernel": (i32, [vp, i32]),
            "fmm_get_m2l_kernel": (i32, [vp]),
            "fmm_set_m2l_shape": (i32, [vp, i32, i32]),
            "fmm_probe_throughput": (i32, [i32, i32, vp, ctypes.POINTER(ctypes.c_double), vp]),
            "fmm_probe_blocks": (i32, []),
            "fmm_get_m2l_shape": (i32, [vp, ctypes.POINTER(i32), ctypes.POINTER(i32)]),
            "fmm_set_near_shape": (i32, [vp, i32]),
            "fmm_get_near_shape": (i32, [vp, ctypes.POINTER(i32)]),
            "fmm_selector_features": (i32, [vp, dbl, vp, vp]),
            "fmm_mlp_create": (i32, [i32, ctypes.POINTER(vp)]),
            "fmm_mlp_destroy": (None, [vp]),
            "fmm_mlp_set_params": (i32, [vp, vp, vp]),
            "fmm_mlp_get_params": (i32, [vp, vp, vp]),
            "fmm_mlp_forward": (i32, [vp, vp, i32, vp, vp]),
            "fmm_mlp_gradients": (i32, [vp, vp, vp, i32, vp, vp, vp]),
            "fmm_mlp_train_step": (i32, [vp, vp, vp, i32, ctypes.c_float, vp, vp]),
            "fmm_select_params": (i32, [vp, vp, i32, vp, vp]),
            "fmm_build_tree": (i32, [vp, vp, vp, vp]),
            "fmm_tree_export": (i32, [vp, vp, vp, vp, vp]),
            "fmm_tree_info": (i32, [vp, ctypes.POINTER(i64), ctypes.POINTER(i32), ctypes.POINTER(i64)]),
            "fmm_tree_destroy": (None, [vp]),
            "fmm_lists_create": (i32, [vp, i64, i64, ctypes.POINTER(vp)]),
            "fmm_interaction_lists": (i32, [vp, vp, dbl, vp]),
            "fmm_lists_set_mode": (i32, [vp, i32]),
            "fmm_lists_import": (i32, [vp, i32, vp, vp, vp, vp, vp]),
            "fmm_validate": (i32, [vp, vp, vp]),
            "fmm_selftest_bounded_wait": (i32, [i64, vp]),
            "fmm_selftest_queue_timeout": (i32, [vp, i64, vp]),
            "fmm_step": (i32, [vp, vp, vp, vp, dbl, vp, ctypes.POINTER(fmm_params), vp, vp]),
            "fmm_build_tree_uniform": (i32, [vp, vp, vp, vp, vp]),
            "fmm_lists_export_exchange": (i32, [vp, i32, vp, vp, ctypes.POINTER(ctypes.c_int64), vp]),
            "fmm_lists_sync": (i32, [vp, vp, ctypes.POINTER(i64), ctypes.POINTER(i64)]),
            "fmm_lists_export": (i32, [vp, vp, vp, vp, vp, vp]),
            "fmm_lists_destroy": (None, [vp]),
            "fmm_evaluate": (i32, [vp, vp, vp, ctypes.POINTER(fmm_params), vp, vp]),
            "fmm_direct": (i32, [vp, vp, vp, i64, vp, i64, vp, vp]),
            "fmm_evaluate_field": (i32, [vp, vp, vp, ctypes.POINTER(fmm_params), vp, vp, vp]),
            "fmm_direct_field": (i32, [vp, vp, vp, i64, vp, i64, vp, vp, vp]),
            "fmm_sync_status": (i32, [vp, vp, vp]),
            "fmm_build_tree_noalloc": (i32, [vp, vp, i64, i32, vp, vp, vp, vp, vp]),
            "fmm_profile_enable": (i32, [i32]),
            "fmm_profile_read": (i32, [vp, vp, i32]),
            "fmm_launch_count": (i64, []),
            "fmm_last_error": (ctypes.c_char_p, []),
        }
        for name, (res, args) in sig.items():
            f = getattr(lib, name)
            f.restype = res
            f.argtypes = args
        _lib = lib
        return lib


def fmm_last_error() -> str:
    return load_library().fmm_last_error().decode()


def _check(rc: int):
    if rc != FMM_OK:
        raise FMMError(rc, fmm_last_error())


def _stream(stream):
    if stream is None:
        return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    if isinstance(stream, torch.cuda.Stream):
        return ctypes.c_void_p(stream.cuda_stream)
    return ctypes.c_void_p(int(stream))


def _need(*specs):
    """(tensor or None, elements, name) triples: the C entry points write through raw pointers
    whose length they cannot see, so a buffer shorter than the call's output is refused here,
    before anything is launched."""
    for t, n, name in specs:
        if t is not None and t.numel() < n:
            raise FMMError(FMM_ERR_ARG, f"{name} has {t.numel()} elements, needs {n}")


def _dev(t: torch.Tensor | None, dtype, n=None, name="tensor"):
    if t is None:
        return None
    if n is not None:
        _need((t, n, name))
    if not t.is_cuda:
        raise FMMError(FMM_ERR_ARG, f"{name} must be a CUDA tensor")
    if t.dtype != dtype:
        raise FMMError(FMM_ERR_ARG, f"{name} must be {dtype}, got {t.dtype}")
    if not t.is_contiguous():
        raise FMMError(FMM_ERR_ARG, f"{name} must be contiguous")
    return ctypes.c_void_p(t.data_ptr())


# ---- entry points, same names as the C ABI ----------------------------------------------------

def fmm_tree_create(n: int, levels: int) -> ctypes.c_void_p:
    h = ctypes.c_void_p()
    _check(load_library().fmm_tree_create(int(n), int(levels), ctypes.byref(h)))
    return h


def fmm_tree_create_batched(ns, levels) -> ctypes.c_void_p:
    """A forest of len(ns) independent instances (instance i: ns[i] points, levels[i] levels)."""
    import numpy as np
    n_arr = np.ascontiguousarray(ns, dtype=np.int64)
    l_arr = np.ascontiguousarray(levels, dtype=np.int32)
    if n_arr.shape != l_arr.shape or n_arr.ndim != 1:
        raise FMMError(FMM_ERR_ARG, "ns and levels must be 1-d sequences of one length")
    h = ctypes.c_void_p()
    _check(load_library().fmm_tree_create_batched(int(n_arr.size), n_arr.ctypes.data_as(ctypes.c_void_p),
                                                  l_arr.ctypes.data_as(ctypes.c_void_p), ctypes.byref(h)))
    return h


def fmm_tree_num_instances(tree) -> int:
    rc = load_library().fmm_tree_num_instances(tree)
    if rc < 0:
        _check(rc)
    return rc


def fmm_tree_instance(tree, i: int) -> dict:
    """Where instance i of a forest lives: p0, n, levels, b0, nbox, lb0."""
    v = [ctypes.c_int64(), ctypes.c_int64(), ctypes.c_int(), ctypes.c_int64(), ctypes.c_int64(), ctypes.c_int64()]
    _check(load_library().fmm_tree_instance(tree, int(i), *[ctypes.byref(a) for a in v]))
    return dict(zip(("p0", "n", "levels", "b0", "nbox", "lb0"), (a.value for a in v)))


def fmm_build_tree(tree, x: torch.Tensor, y: torch.Tensor, stream=None):
    n = fmm_tree_info(tree)[0]
    _check(load_library().fmm_build_tree(tree, _dev(x, torch.float64, n, "x"),
                                         _dev(y, torch.float64, n, "y"), _stream(stream)))


def fmm_build_tree_uniform(tree, x: torch.Tensor, y: torch.Tensor, root=None, stream=None):
    """The uniform-grid mesh (square root, geometric quadrants) in place of the median tree, for
    the adaptive-vs-uniform comparison; ``root`` = (x0, y0, side) fixes the root square (default:
    the bounding square).  Synchronises the stream."""
    n = fmm_tree_info(tree)[0]
    r = None if root is None else (ctypes.c_double * 3)(*[float(v) for v in root])
    _check(load_library().fmm_build_tree_uniform(tree, _dev(x, torch.float64, n, "x"),
                                                 _dev(y, torch.float64, n, "y"),
                                                 None if r is None else ctypes.cast(r, ctypes.c_void_p),
                                                 _stream(stream)))


FMM_NOALLOC_MAX_POINTS = 65536
FMM_NOALLOC_MAX_LEVELS = 7


def fmm_build_tree_noalloc(x, y, levels: int, perm, rects, leaf_begin, status=None, stream=None):
    """Tree build for callers that cannot allocate device memory: the outputs are the caller's
    tensors, every intermediate lives in the library's fixed device array (n <= 65536,
    levels <= 7).  Calls on one device must not overlap in time."""
    n, L = x.numel(), int(levels)
    nbox = (4 ** (L + 1) - 1) // 3 if 0 <= L <= FMM_NOALLOC_MAX_LEVELS else 0
    _need((y, n, "y"), (perm, n, "perm"), (rects, 4 * nbox, "rects"),
          (leaf_begin, 4 ** L + 1 if nbox else 0, "leaf_begin"))
    args = (_dev(x, torch.float64, n, "x"), _dev(y, torch.float64, n, "y"), n, L,
            _dev(perm, torch.int32, n, "perm"), _dev(rects, torch.float64, 4 * nbox, "rects"),
            _dev(leaf_begin, torch.int32, 4 ** L + 1 if nbox else 0, "leaf_begin"),
            _dev(status, torch.int32, 1, "status"), _stream(stream))
    _check(load_library().fmm_build_tree_noalloc(*args))


def fmm_tree_export(tree, perm=None, rects=None, leaf_begin=None, stream=None):
    n, L, nbox = fmm_tree_info(tree)
    last = fmm_tree_instance(tree, fmm_tree_num_instances(tree) - 1)
    nlb = last["lb0"] + 4 ** last["levels"] + 1  # every instance's 4^L_i + 1 offsets
    _need((perm, n, "perm"), (rects, 4 * nbox, "rects"), (leaf_begin, nlb, "leaf_begin"))
    args = (tree, _dev(perm, torch.int32, n, "perm"), _dev(rects, torch.float64, 4 * nbox, "rects"),
            _dev(leaf_begin, torch.int32, 4 ** L + 1, "leaf_begin"), _stream(stream))
    _check(load_library().fmm_tree_export(*args))


def fmm_tree_info(tree):
    n, L, nb = ctypes.c_int64(), ctypes.c_int(), ctypes.c_int64()
    _check(load_library().fmm_tree_info(tree, ctypes.byref(n), ctypes.byref(L), ctypes.byref(nb)))
    return n.value, L.value, nb.value


def fmm_tree_destroy(tree):
    if tree:
        load_library().fmm_tree_destroy(tree)


def fmm_lists_create(tree, weak_capacity: int = 0, strong_capacity: int = 0) -> ctypes.c_void_p:
    h = ctypes.c_void_p()
    _check(load_library().fmm_lists_create(tree, int(weak_capacity), int(strong_capacity), ctypes.byref(h)))
    return h


def fmm_lists_create_batched(tree, weak_capacity, strong_capacity) -> ctypes.c_void_p:
    import numpy as np
    w = np.ascontiguousarray(weak_capacity, dtype=np.int64)
    st = np.ascontiguousarray(strong_capacity, dtype=np.int64)
    ni = fmm_tree_num_instances(tree)
    if w.shape != (ni,) or st.shape != (ni,):
        raise FMMError(FMM_ERR_ARG, f"capacities need {ni} entries each")
    h = ctypes.c_void_p()
    _check(load_library().fmm_lists_create_batched(tree, w.ctypes.data_as(ctypes.c_void_p),
                                                   st.ctypes.data_as(ctypes.c_void_p), ctypes.byref(h)))
    return h


def fmm_lists_counts(lists, n_inst: int, stream=None, check: bool = True):
    """Per-instance (weak, strong) entry counts; with check=False a capacity overflow is
    returned as the third value instead of raised."""
    import numpy as np
    w = np.zeros(n_inst, np.int64)
    st = np.zeros(n_inst, np.int64)
    rc = load_library().fmm_lists_counts(lists, _stream(stream), w.ctypes.data_as(ctypes.c_void_p),
                                         st.ctypes.data_as(ctypes.c_void_p))
    if check:
        _check(rc)
        return w, st
    if rc not in (FMM_OK, FMM_ERR_CAPACITY):
        _check(rc)
    return w, st, rc == FMM_ERR_CAPACITY


FMM_LISTS_PLAIN, FMM_LISTS_PARENTS, FMM_LISTS_EXCHANGE = 0, 1, 2
FMM_PARENT_FLAG, FMM_SWAP_M2P = 0x40000000, 0x20000000


def fmm_lists_set_mode(lists, mode: int):
    """Bits of Section 4's optional optimisations: FMM_LISTS_PARENTS (four weak siblings become
    their parent where the criterion allows), FMM_LISTS_EXCHANGE (finest-level role exchange:
    P2L / M2P for strongly coupled leaves of different radii)."""
    _check(load_library().fmm_lists_set_mode(lists, int(mode)))


def fmm_lists_export_exchange(lists, i: int, xoff=None, xidx=None, stream=None) -> int:
    """Instance i's exchange lists into device int32 buffers (either may be None); returns the
    number of entries."""
    n = ctypes.c_int64()
    _check(load_library().fmm_lists_export_exchange(lists, int(i), _dev(xoff, torch.int32, None, "xoff"),
                                                    _dev(xidx, torch.int32, None, "xidx"), ctypes.byref(n),
                                                    _stream(stream)))
    return n.value


def _lists_mode(parents: bool, exchange: bool) -> int:
    return (FMM_LISTS_PARENTS if parents else 0) | (FMM_LISTS_EXCHANGE if exchange else 0)


def fmm_interaction_lists(tree, lists, theta: float, stream=None):
    _check(load_library().fmm_interaction_lists(tree, lists, float(theta), _stream(stream)))


def fmm_lists_sync(lists, stream=None):
    w, s = ctypes.c_int64(), ctypes.c_int64()
    _check(load_library().fmm_lists_sync(lists, _stream(stream), ctypes.byref(w), ctypes.byref(s)))
    return w.value, s.value


def fmm_lists_import(lists, i: int, woff, widx, soff, sidx, stream=None):
    """Instance i's lists from device int32 arrays in the export layout (then fmm_validate)."""
    _check(load_library().fmm_lists_import(lists, int(i), _dev(woff, torch.int32, None, "woff"),
                                           _dev(widx, torch.int32, None, "widx"), _dev(soff, torch.int32, None, "soff"),
                                           _dev(sidx, torch.int32, None, "sidx"), _stream(stream)))


def fmm_selftest_queue_timeout(tree, tries: int = 4096, stream=None):
    """The queued upward pass with a producer missing from the queue: raises
    FMMError(FMM_ERR_TIMEOUT) when the bounded waits give up, as designed."""
    _check(load_library().fmm_selftest_queue_timeout(tree, int(tries), _stream(stream)))


def fmm_selftest_bounded_wait(tries: int = 4096, stream=None):
    """The bounded device wait on an mbarrier nothing completes: raises FMMError(FMM_ERR_TIMEOUT)
    when it gives up, as designed."""
    _check(load_library().fmm_selftest_bounded_wait(int(tries), _stream(stream)))


def fmm_validate(tree, lists=None, stream=None):
    """Structural checks of a built tree and its lists; raises FMMError naming a failed check."""
    _check(load_library().fmm_validate(tree, lists, _stream(stream)))


def fmm_lists_export(lists, woff, widx, soff, sidx, stream=None):
    _check(load_library().fmm_lists_export(lists, _dev(woff, torch.int32, None, "woff"),
                                           _dev(widx, torch.int32, None, "widx"),
                                           _dev(soff, torch.int32, None, "soff"),
                                           _dev(sidx, torch.int32, None, "sidx"), _stream(stream)))


def fmm_lists_export_instance(lists, i: int, woff, widx, soff, sidx, stream=None):
    _check(load_library().fmm_lists_export_instance(lists, int(i), _dev(woff, torch.int32, None, "woff"),
                                                    _dev(widx, torch.int32, None, "widx"),
                                                    _dev(soff, torch.int32, None, "soff"),
                                                    _dev(sidx, torch.int32, None, "sidx"), _stream(stream)))


def fmm_lists_destroy(lists):
    if lists:
        load_library().fmm_lists_destroy(lists)


def fmm_evaluate(tree, lists, q: torch.Tensor, p: int, mode: int, phi: torch.Tensor, tol: float = 1e-6,
                 stream=None):
    n = fmm_tree_info(tree)[0]
    prm = fmm_params(int(p), int(mode), float(tol))
    _check(load_library().fmm_evaluate(tree, lists, _dev(q, torch.float64, n, "q"), ctypes.byref(prm),
                                       _dev(phi, torch.float64, n, "phi"), _stream(stream)))


def fmm_autotune(tree, lists, q: torch.Tensor, p: int, mode: int, phi: torch.Tensor, tol: float = 1e-6,
                 stream=None):
    """Time complete evaluations over a ladder of grid sizes and keep the fastest; returns the
    chosen (M2L, near-field) blocks per instance."""
    n = fmm_tree_info(tree)[0]
    prm = fmm_params(int(p), int(mode), float(tol))
    a, b = ctypes.c_int(), ctypes.c_int()
    _check(load_library().fmm_autotune(tree, lists, _dev(q, torch.float64, n, "q"), ctypes.byref(prm),
                                       _dev(phi, torch.float64, n, "phi"), _stream(stream),
                                       ctypes.byref(a), ctypes.byref(b)))
    return a.value, b.value


def fmm_set_launch(tree, m2l_blocks: int = 0, p2p_blocks: int = 0):
    _check(load_library().fmm_set_launch(tree, int(m2l_blocks), int(p2p_blocks)))


FMM_MLP_IN, FMM_MLP_HIDDEN, FMM_MLP_OUT, FMM_MLP_PARAMS = 64, 128, 225, 53857
FMM_SEL_LMIN, FMM_SEL_LMAX, FMM_SEL_PMIN, FMM_SEL_PMAX, FMM_SEL_NP = 4, 12, 8, 32, 25


def fmm_selector_features(tree, tol: float, out: torch.Tensor, stream=None):
    """Selector inputs of every instance of a built tree: out[n_inst][64] (CUDA float32)."""
    ni = fmm_tree_num_instances(tree)
    _check(load_library().fmm_selector_features(tree, float(tol), _dev(out, torch.float32, 64 * ni, "features"),
                                                _stream(stream)))


def fmm_mlp_create(batch_max: int) -> ctypes.c_void_p:
    h = ctypes.c_void_p()
    _check(load_library().fmm_mlp_create(int(batch_max), ctypes.byref(h)))
    return h


def fmm_mlp_destroy(m):
    if m:
        load_library().fmm_mlp_destroy(m)


def fmm_mlp_set_params(m, params: torch.Tensor, stream=None):
    _check(load_library().fmm_mlp_set_params(m, _dev(params, torch.float32, FMM_MLP_PARAMS, "params"),
                                             _stream(stream)))


def fmm_mlp_get_params(m, out: torch.Tensor, stream=None):
    _check(load_library().fmm_mlp_get_params(m, _dev(out, torch.float32, FMM_MLP_PARAMS, "params"),
                                             _stream(stream)))


def fmm_mlp_forward(m, X: torch.Tensor, prob: torch.Tensor, stream=None):
    B = X.shape[0]
    _check(load_library().fmm_mlp_forward(m, _dev(X, torch.float32, 64 * B, "X"), B,
                                          _dev(prob, torch.float32, 225 * B, "prob"), _stream(stream)))


def fmm_mlp_gradients(m, X: torch.Tensor, labels: torch.Tensor, grad=None, loss=None, stream=None):
    B = X.shape[0]
    _check(load_library().fmm_mlp_gradients(m, _dev(X, torch.float32, 64 * B, "X"),
                                            _dev(labels, torch.int32, B, "labels"), B,
                                            _dev(grad, torch.float32, FMM_MLP_PARAMS, "grad"),
                                            _dev(loss, torch.float32, 1, "loss"), _stream(stream)))


def fmm_mlp_train_step(m, X: torch.Tensor, labels: torch.Tensor, lr: float, loss=None, stream=None):
    B = X.shape[0]
    _check(load_library().fmm_mlp_train_step(m, _dev(X, torch.float32, 64 * B, "X"),
                                             _dev(labels, torch.int32, B, "labels"), B, float(lr),
                                             _dev(loss, torch.float32, 1, "loss"), _stream(stream)))


def fmm_select_params(m, features: torch.Tensor, out: torch.Tensor, stream=None):
    """out[B][2] (CUDA int32) = (levels, p) chosen for each feature vector."""
    B = features.shape[0]
    _check(load_library().fmm_select_params(m, _dev(features, torch.float32, 64 * B, "features"), B,
                                            _dev(out, torch.int32, 2 * B, "out"), _stream(stream)))


FMM_M2L_AUTO, FMM_M2L_SIMT, FMM_M2L_TENSOR = 0, 1, 2


def fmm_set_m2l_kernel(tree, kind: int):
    """Binary32 M2L by order (0, default), on the SIMT units (1) or on the tensor cores (2)."""
    _check(load_library().fmm_set_m2l_kernel(tree, int(kind)))


def fmm_get_m2l_kernel(tree) -> int:
    rc = load_library().fmm_get_m2l_kernel(tree)
    if rc < 0:
        _check(rc)
    return rc


FMM_PROBE_FFMA, FMM_PROBE_LG2, FMM_PROBE_DFMA = 0, 1, 2


def fmm_probe_blocks() -> int:
    rc = load_library().fmm_probe_blocks()
    if rc < 0:
        _check(rc)
    return rc


def fmm_probe_throughput(kind: int, iters: int = 4096, reps: int = 3) -> float:
    """Measured throughput of one unit (operations per second; flop for the FMA probes): the
    best of `reps` timed launches of the library's probe kernel on the current stream."""
    lib = load_library()
    nb = fmm_probe_blocks()
    out = torch.empty(nb * 256, dtype=torch.float32, device="cuda")
    ops = ctypes.c_double()
    stream = torch.cuda.current_stream()
    _check(lib.fmm_probe_throughput(int(kind), int(iters), ctypes.c_void_p(out.data_ptr()), ctypes.byref(ops),
                                    _stream(None)))  # warm-up
    best = float("inf")
    for _ in range(reps):
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        _check(lib.fmm_probe_throughput(int(kind), int(iters), ctypes.c_void_p(out.data_ptr()),
                                        ctypes.byref(ops), _stream(None)))
        b.record(stream)
        b.synchronize()
        best = min(best, a.elapsed_time(b) * 1e-3)
    return ops.value / best


def fmm_set_m2l_shape(tree, chunk: int = 0, stages: int = 0):
    """Tensor-core M2L tile shape: consecutive weak entries per row (0: default) and TMEM
    accumulator stages (1, 2; 0: by order)."""
    _check(load_library().fmm_set_m2l_shape(tree, int(chunk), int(stages)))


def fmm_get_m2l_shape(tree):
    c, st = ctypes.c_int(), ctypes.c_int()
    _check(load_library().fmm_get_m2l_shape(tree, ctypes.byref(c), ctypes.byref(st)))
    return c.value, st.value


def fmm_set_near_shape(tree, targets: int = 0):
    """binary32 near field: targets per lane (2, 4; 0: default)."""
    _check(load_library().fmm_set_near_shape(tree, int(targets)))


def fmm_get_near_shape(tree):
    t = ctypes.c_int()
    _check(load_library().fmm_get_near_shape(tree, ctypes.byref(t)))
    return t.value


def fmm_step(tree, lists, x: torch.Tensor, y: torch.Tensor, theta: float, q: torch.Tensor, p: int, mode: int,
             phi: torch.Tensor, tol: float = 1e-6, stream=None):
    """Tree, lists and evaluation in one call, the independent parts overlapped on the tree's
    second stream (capturable into a CUDA graph after a first call)."""
    n = fmm_tree_info(tree)[0]
    prm = fmm_params(int(p), int(mode), float(tol))
    _check(load_library().fmm_step(tree, lists, _dev(x, torch.float64, n, "x"), _dev(y, torch.float64, n, "y"),
                                   float(theta), _dev(q, torch.float64, n, "q"), ctypes.byref(prm),
                                   _dev(phi, torch.float64, n, "phi"), _stream(stream)))


def fmm_evaluate_field(tree, lists, q: torch.Tensor, p: int, mode: int, fre: torch.Tensor, fim: torch.Tensor,
                       tol: float = 1e-6, stream=None):
    """The complex field F_i = sum_{j != i} -q_j / (z_i - z_j): real part into fre, imaginary
    part into fim (CUDA float64, input order)."""
    n = fmm_tree_info(tree)[0]
    prm = fmm_params(int(p), int(mode), float(tol))
    _check(load_library().fmm_evaluate_field(tree, lists, _dev(q, torch.float64, n, "q"), ctypes.byref(prm),
                                             _dev(fre, torch.float64, n, "fre"), _dev(fim, torch.float64, n, "fim"),
                                             _stream(stream)))


def fmm_direct_field(x, y, q, targets, fre, fim, stream=None):
    n = x.numel()
    m = targets.numel()
    _check(load_library().fmm_direct_field(_dev(x, torch.float64, n, "x"), _dev(y, torch.float64, n, "y"),
                                           _dev(q, torch.float64, n, "q"), n,
                                           _dev(targets, torch.int64, m, "targets"), m,
                                           _dev(fre, torch.float64, m, "fre"), _dev(fim, torch.float64, m, "fim"),
                                           _stream(stream)))


def fmm_direct(x, y, q, targets, phi, stream=None):
    n = x.numel()
    m = targets.numel()
    _check(load_library().fmm_direct(_dev(x, torch.float64, n, "x"), _dev(y, torch.float64, n, "y"),
                                     _dev(q, torch.float64, n, "q"), n,
                                     _dev(targets, torch.int64, m, "targets"), m,
                                     _dev(phi, torch.float64, m, "phi"), _stream(stream)))


def fmm_sync_status(tree, lists=None, stream=None):
    _check(load_library().fmm_sync_status(tree, lists, _stream(stream)))


STAGES = ("tree_sort", "tree_split", "tree_finish", "lists", "gather", "p2m", "m2m", "m2l", "l2l",
          "leaf", "near", "exchange")


def fmm_profile_enable(on: bool = True):
    _check(load_library().fmm_profile_enable(1 if on else 0))


def fmm_profile_read():
    """Per-stage (milliseconds, count) recorded since the last read."""
    import numpy as np
    ms = np.zeros(len(STAGES), np.float64)
    cnt = np.zeros(len(STAGES), np.int64)
    rc = load_library().fmm_profile_read(ms.ctypes.data_as(ctypes.c_void_p),
                                         cnt.ctypes.data_as(ctypes.c_void_p), len(STAGES))
    if rc < 0:
        _check(rc)
    return {k: (float(ms[i]), int(cnt[i])) for i, k in enumerate(STAGES)}


def fmm_launch_count() -> int:
    return int(load_library().fmm_launch_count())


# ---- convenience ---------------------------------------------------------------------------

def _export_exchange(lists, i, nbox, device):
    xoff = torch.empty(nbox + 1, dtype=torch.int32, device=device)
    nx = fmm_lists_export_exchange(lists, i, xoff, None)
    xidx = torch.empty(max(nx, 1), dtype=torch.int32, device=device)
    fmm_lists_export_exchange(lists, i, None, xidx)
    torch.cuda.synchronize(device)
    return xoff, xidx[:nx]


class FMM:
    """One point set: its tree, its interaction lists and any number of evaluations.

    >>> f = FMM(x, y, levels=8, theta=0.5)          # x, y: CUDA float64
    >>> phi = f.evaluate(q, p=20, mode="mixed")      # potentials in input order
    """

    def __init__(self, x: torch.Tensor, y: torch.Tensor, levels: int, theta: float = 0.5,
                 weak_capacity: int = 0, strong_capacity: int = 0, check: bool = True, parents: bool = False,
                 exchange: bool = False, mesh: str = "adaptive", root=None):
        if mesh not in ("adaptive", "uniform"):
            raise FMMError(FMM_ERR_ARG, f"mesh must be 'adaptive' or 'uniform', not {mesh!r}")
        self.mesh = mesh
        self.root = root  # uniform mesh: (x0, y0, side) or None for the bounding square
        self.n = x.numel()
        self.levels = levels
        self.theta = theta
        self.device = x.device
        self.mode = _lists_mode(parents, exchange)
        self.tree = fmm_tree_create(self.n, levels)
        self.lists = None
        try:
            self.lists = fmm_lists_create(self.tree, weak_capacity, strong_capacity)
            if self.mode:
                fmm_lists_set_mode(self.lists, self.mode)
            self.rebuild(x, y, check=check)
        except Exception:
            self.close()
            raise

    def rebuild(self, x, y, theta=None, check: bool = True):
        """Rebuild tree and lists for new coordinates (same n and levels); grows the list
        capacity and retries when the lists overflow."""
        if theta is not None:
            self.theta = theta
        if self.mesh == "uniform":
            fmm_build_tree_uniform(self.tree, x, y, self.root)
        else:
            fmm_build_tree(self.tree, x, y)
        fmm_interaction_lists(self.tree, self.lists, self.theta)
        if check:
            try:
                self.counts = fmm_lists_sync(self.lists)
            except FMMError as e:
                if e.code != FMM_ERR_CAPACITY:
                    raise
                w, s = self._needed()
                if self.mode & FMM_LISTS_EXCHANGE:
                    s = max(s, fmm_lists_export_exchange(self.lists, 0))  # the exchange lists share it
                fmm_lists_destroy(self.lists)
                self.lists = None
                self.lists = fmm_lists_create(self.tree, 2 * w + 1024, 2 * s + 1024)
                if self.mode:
                    fmm_lists_set_mode(self.lists, self.mode)
                return self.rebuild(x, y, check=check)
            fmm_sync_status(self.tree, self.lists)

    def _needed(self):
        nbox = fmm_tree_info(self.tree)[2]
        woff = torch.empty(nbox + 1, dtype=torch.int32, device=self.device)
        soff = torch.empty(nbox + 1, dtype=torch.int32, device=self.device)
        fmm_lists_export(self.lists, woff, None, soff, None)
        torch.cuda.synchronize(self.device)
        return int(woff[-1]), int(soff[-1])

    def evaluate(self, q, p: int, mode: str | int = "mixed", tol: float = 1e-6, out=None,
                 check: bool = True):
        m = {"fp64": FMM_MODE_FP64, "mixed": FMM_MODE_MIXED, "split": FMM_MODE_SPLIT}.get(mode, mode)
        phi = out if out is not None else torch.empty(self.n, dtype=torch.float64, device=self.device)
        fmm_evaluate(self.tree, self.lists, q, p, m, phi, tol)
        if check:
            fmm_sync_status(self.tree, self.lists)
        return phi

    def evaluate_field(self, q, p: int, mode: str | int = "mixed", tol: float = 1e-6, check: bool = True):
        """The complex field F_i = sum_{j != i} -q_j / (z_i - z_j) (complex128 CUDA tensor)."""
        m = {"fp64": FMM_MODE_FP64, "mixed": FMM_MODE_MIXED, "split": FMM_MODE_SPLIT}.get(mode, mode)
        fre = torch.empty(self.n, dtype=torch.float64, device=self.device)
        fim = torch.empty(self.n, dtype=torch.float64, device=self.device)
        fmm_evaluate_field(self.tree, self.lists, q, p, m, fre, fim, tol)
        if check:
            fmm_sync_status(self.tree, self.lists)
        return torch.complex(fre, fim)

    def export_tree(self):
        n, L, nbox = fmm_tree_info(self.tree)
        perm = torch.empty(n, dtype=torch.int32, device=self.device)
        rects = torch.empty((nbox, 4), dtype=torch.float64, device=self.device)
        lb = torch.empty(4 ** L + 1, dtype=torch.int32, device=self.device)
        fmm_tree_export(self.tree, perm, rects, lb)
        return perm, rects, lb

    def export_lists(self):
        nbox = fmm_tree_info(self.tree)[2]
        w, s = fmm_lists_sync(self.lists)
        woff = torch.empty(nbox + 1, dtype=torch.int32, device=self.device)
        soff = torch.empty(nbox + 1, dtype=torch.int32, device=self.device)
        widx = torch.empty(max(w, 1), dtype=torch.int32, device=self.device)
        sidx = torch.empty(max(s, 1), dtype=torch.int32, device=self.device)
        fmm_lists_export(self.lists, woff, widx, soff, sidx)
        torch.cuda.synchronize(self.device)
        return woff, widx[:w], soff, sidx[:s]

    def export_exchange(self):
        """The role-exchange lists (xoff over all boxes, xidx) of a build with exchange=True."""
        return _export_exchange(self.lists, 0, fmm_tree_info(self.tree)[2], self.device)

    def close(self):
        if self.lists is not None:
            fmm_lists_destroy(self.lists)
            self.lists = None
        if self.tree is not None:
            fmm_tree_destroy(self.tree)
            self.tree = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class FMMBatch:
    """Many independent point sets evaluated together: one forest tree, one set of lists, and
    every launch covering all instances.  Coordinates, strengths and potentials are the
    instances' arrays concatenated in instance order.

    >>> b = FMMBatch(x, y, sizes=[1000, 50000], levels=[3, 6], theta=0.5)
    >>> phi = b.evaluate(q, p=16)
    """

    def __init__(self, x: torch.Tensor, y: torch.Tensor, sizes, levels, theta: float = 0.5,
                 check: bool = True, weak_per_box: int = 48, strong_per_box: int = 24, parents: bool = False,
                 exchange: bool = False, mesh: str = "adaptive", root=None):
        if mesh not in ("adaptive", "uniform"):
            raise FMMError(FMM_ERR_ARG, f"mesh must be 'adaptive' or 'uniform', not {mesh!r}")
        self.mesh = mesh
        self.root = root
        self.sizes = [int(v) for v in sizes]
        self.levels = [int(v) for v in levels]
        self.n = sum(self.sizes)
        self.n_inst = len(self.sizes)
        self.theta = theta
        self.device = x.device
        self.tree = fmm_tree_create_batched(self.sizes, self.levels)
        self.lists = None
        self.inst = [fmm_tree_instance(self.tree, i) for i in range(self.n_inst)]
        try:
            nb = [d["nbox"] for d in self.inst]
            self.mode = _lists_mode(parents, exchange)
            self.lists = fmm_lists_create_batched(self.tree, [weak_per_box * v for v in nb],
                                                  [strong_per_box * v for v in nb])
            if self.mode:
                fmm_lists_set_mode(self.lists, self.mode)
            self.rebuild(x, y, check=check)
        except Exception:
            self.close()
            raise

    def rebuild(self, x, y, theta=None, check: bool = True):
        """Rebuild for new coordinates (same sizes and levels); regrows the capacity of every
        instance whose lists overflowed and rebuilds."""
        if theta is not None:
            self.theta = theta
        if self.mesh == "uniform":
            fmm_build_tree_uniform(self.tree, x, y, self.root)
        else:
            fmm_build_tree(self.tree, x, y)
        fmm_interaction_lists(self.tree, self.lists, self.theta)
        if check:
            w, s, over = fmm_lists_counts(self.lists, self.n_inst, check=False)
            if over:
                nb = [d["nbox"] for d in self.inst]
                if self.mode & FMM_LISTS_EXCHANGE:  # the exchange lists share the strong capacity
                    s = [max(int(a), fmm_lists_export_exchange(self.lists, i)) for i, a in enumerate(s)]
                fmm_lists_destroy(self.lists)
                self.lists = None
                # counts of an instance that overflowed are lower bounds: at least double it
                self.lists = fmm_lists_create_batched(self.tree, [max(2 * int(a) + 64, 16 * b) for a, b in zip(w, nb)],
                                                      [max(2 * int(a) + 64, 8 * b) for a, b in zip(s, nb)])
                if self.mode:
                    fmm_lists_set_mode(self.lists, self.mode)
                return self.rebuild(x, y, check=check)
            self.counts = (w, s)
            fmm_sync_status(self.tree, self.lists)

    def evaluate(self, q, p: int, mode: str | int = "mixed", tol: float = 1e-6, out=None,
                 check: bool = True):
        m = {"fp64": FMM_MODE_FP64, "mixed": FMM_MODE_MIXED, "split": FMM_MODE_SPLIT}.get(mode, mode)
        phi = out if out is not None else torch.empty(self.n, dtype=torch.float64, device=self.device)
        fmm_evaluate(self.tree, self.lists, q, p, m, phi, tol)
        if check:
            fmm_sync_status(self.tree, self.lists)
        return phi

    def evaluate_field(self, q, p: int, mode: str | int = "mixed", tol: float = 1e-6, check: bool = True):
        m = {"fp64": FMM_MODE_FP64, "mixed": FMM_MODE_MIXED, "split": FMM_MODE_SPLIT}.get(mode, mode)
        fre = torch.empty(self.n, dtype=torch.float64, device=self.device)
        fim = torch.empty(self.n, dtype=torch.float64, device=self.device)
        fmm_evaluate_field(self.tree, self.lists, q, p, m, fre, fim, tol)
        if check:
            fmm_sync_status(self.tree, self.lists)
        return torch.complex(fre, fim)

    def autotune(self, q, p: int, mode: str | int = "mixed", tol: float = 1e-6):
        m = {"fp64": FMM_MODE_FP64, "mixed": FMM_MODE_MIXED, "split": FMM_MODE_SPLIT}.get(mode, mode)
        phi = torch.empty(self.n, dtype=torch.float64, device=self.device)
        return fmm_autotune(self.tree, self.lists, q, p, m, phi, tol)

    def export_exchange(self, i: int):
        """Instance i's role-exchange lists (xoff over its boxes, xidx)."""
        return _export_exchange(self.lists, i, self.inst[i]["nbox"], self.device)

    def export_instance(self, i: int):
        """perm, rects, leaf_begin and the lists (woff, widx, soff, sidx) of instance i."""
        d = self.inst[i]
        n, L, nbox = fmm_tree_info(self.tree)
        perm = torch.empty(n, dtype=torch.int32, device=self.device)
        rects = torch.empty((nbox, 4), dtype=torch.float64, device=self.device)
        nlb = sum(4 ** v + 1 for v in self.levels)
        lb = torch.empty(nlb, dtype=torch.int32, device=self.device)
        fmm_tree_export(self.tree, perm, rects, lb)
        w, s = fmm_lists_counts(self.lists, self.n_inst)
        woff = torch.empty(d["nbox"] + 1, dtype=torch.int32, device=self.device)
        soff = torch.empty(d["nbox"] + 1, dtype=torch.int32, device=self.device)
        widx = torch.empty(max(int(w[i]), 1), dtype=torch.int32, device=self.device)
        sidx = torch.empty(max(int(s[i]), 1), dtype=torch.int32, device=self.device)
        fmm_lists_export_instance(self.lists, i, woff, widx, soff, sidx)
        torch.cuda.synchronize(self.device)
        p0, lb0 = d["p0"], d["lb0"]
        return (perm[p0:p0 + d["n"]], rects[d["b0"]:d["b0"] + d["nbox"]],
                lb[lb0:lb0 + 4 ** d["levels"] + 1], woff, widx[:int(w[i])], soff, sidx[:int(s[i])])

    def close(self):
        if self.lists is not None:
            fmm_lists_destroy(self.lists)
            self.lists = None
        if self.tree is not None:
            fmm_tree_destroy(self.tree)
            self.tree = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
