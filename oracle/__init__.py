"""Plain FP64 CPU oracle for the asymmetric adaptive 2D FMM (Engblom, "On well-separated sets
and fast multipole methods").

TEST INFRASTRUCTURE ONLY: the test suite, ``__graft_entry__.smoke()`` and the CPU-baseline leg
of ``bench.py`` are the only code allowed to import this package.  It never imports the CUDA
package and the CUDA package never imports it.

The arithmetic lives in ``fmm_oracle.c`` (compiled with ``-ffp-contract=off`` so that no
multiply-add is fused); this module only compiles it and marshals numpy arrays:

* :func:`tree`       -- median-split mesh (Section 4, Fig. 1.1, Fig. 4.1)
* :func:`tree_uniform` -- the uniform-grid mesh of the comparison in Section 5
* :func:`lists`      -- strong/weak connectivity with the theta-criterion (Section 4, Crit. 2.1)
* :func:`fmm`        -- the whole method, P2M .. P2P, unscaled textbook expansions (Section 5)
* :func:`direct`     -- the O(N^2) definition, Eq. (1.1)
* :func:`fmm_field`, :func:`direct_field` -- the complex field -q_j / (z_i - z_j) of Section 5's
  first experiment, by the method and by direct summation
* :func:`p2m`, :func:`m2m`, :func:`m2l`, :func:`l2l`, :func:`l2p`, :func:`m2p`, :func:`p2l` -- one
  operator at a time, for the pins.
* :mod:`oracle.mlp`  -- FP64 reference of the parameter-selector network.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "fmm_oracle.c")
_SRCS = [_SRC, os.path.join(_HERE, "mlp_oracle.c")]
_SO = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile ``fmm_oracle.c`` and ``mlp_oracle.c`` into ``liboracle.so`` next to them (plain
    gcc, no GPU)."""
    if not force and os.path.exists(_SO) and all(os.path.getmtime(_SO) >= os.path.getmtime(f) for f in _SRCS):
        return _SO
    base = ["gcc", "-O2", "-fPIC", "-shared", "-ffp-contract=off", "-fcx-fortran-rules",
            "-fno-fast-math", "-o", _SO + ".tmp", *_SRCS, "-lm"]
    try:
        subprocess.run(base[:1] + ["-fopenmp"] + base[1:], check=True, capture_output=True)
    except subprocess.CalledProcessError:
        subprocess.run(base, check=True, capture_output=True)  # no OpenMP: single thread
    os.replace(_SO + ".tmp", _SO)
    return _SO


def _load():
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        lib = ctypes.CDLL(build())
        i64, i32, dbl, vp = ctypes.c_int64, ctypes.c_int, ctypes.c_double, ctypes.c_void_p
        lib.orc_nbox.restype = i64
        lib.orc_nbox.argtypes = [i32]
        lib.orc_tree.restype = i32
        lib.orc_tree.argtypes = [i64, vp, vp, i32, vp, vp, vp]
        lib.orc_tree_uniform.restype = i32
        lib.orc_tree_uniform.argtypes = [i64, vp, vp, i32, vp, vp, vp, vp]
        lib.orc_fmm_root.restype = i32
        lib.orc_fmm_root.argtypes = [i64, vp, vp, vp, i32, i32, dbl, i32, vp, vp]
        lib.orc_geometry.restype = None
        lib.orc_geometry.argtypes = [i64, vp, vp, vp]
        lib.orc_theta_weak.restype = i32
        lib.orc_theta_weak.argtypes = [dbl] * 7
        lib.orc_lists_build.restype = vp
        lib.orc_lists_build.argtypes = [i32, vp, dbl]
        lib.orc_lists_total.restype = i64
        lib.orc_lists_total.argtypes = [vp, i32]
        lib.orc_lists_copy.restype = None
        lib.orc_lists_copy.argtypes = [vp, i32, vp, vp]
        lib.orc_lists_free.restype = None
        lib.orc_lists_free.argtypes = [vp]
        lib.orc_p2m.restype = None
        lib.orc_p2m.argtypes = [i64, vp, vp, vp, dbl, dbl, i32, vp]
        for name in ("orc_m2m", "orc_m2l", "orc_l2l"):
            getattr(lib, name).restype = None
            getattr(lib, name).argtypes = [vp, dbl, dbl, i32, vp]
        for name in ("orc_l2p", "orc_m2p"):
            getattr(lib, name).restype = dbl
            getattr(lib, name).argtypes = [vp, dbl, dbl, i32]
        lib.orc_direct.restype = None
        lib.orc_direct.argtypes = [i64, vp, vp, vp, i64, vp, vp, i32]
        lib.orc_fmm.restype = i32
        lib.orc_fmm.argtypes = [i64, vp, vp, vp, i32, i32, dbl, vp, vp, vp]
        lib.orc_fmm_ex.restype = i32
        lib.orc_fmm_ex.argtypes = [i64, vp, vp, vp, i32, i32, dbl, i32, vp]
        lib.orc_lists_merge_parents.restype = None
        lib.orc_lists_merge_parents.argtypes = [vp, vp, dbl]
        lib.orc_lists_swap_leaves.restype = None
        lib.orc_lists_swap_leaves.argtypes = [vp, vp, dbl]
        lib.orc_theta_swapped.restype = i32
        lib.orc_theta_swapped.argtypes = [dbl] * 7
        lib.orc_p2l.restype = None
        lib.orc_p2l.argtypes = [i64, vp, vp, vp, dbl, dbl, i32, vp]
        lib.orc_fmm_field_ex.restype = i32
        lib.orc_fmm_field_ex.argtypes = [i64, vp, vp, vp, i32, i32, dbl, i32, vp, vp]
        lib.orc_fmm_field.restype = i32
        lib.orc_fmm_field.argtypes = [i64, vp, vp, vp, i32, i32, dbl, vp, vp]
        lib.orc_direct_field.restype = None
        lib.orc_direct_field.argtypes = [i64, vp, vp, vp, i64, vp, vp, vp, i32]
        lib.orc_mlp_nparams.restype = ctypes.c_long
        lib.orc_mlp_nparams.argtypes = []
        lib.orc_mlp_forward.restype = None
        lib.orc_mlp_forward.argtypes = [vp, vp, i32, vp]
        lib.orc_mlp_loss_grad.restype = dbl
        lib.orc_mlp_loss_grad.argtypes = [vp, vp, vp, i32, vp]
        lib.orc_features.restype = None
        lib.orc_features.argtypes = [vp, i32, i64, dbl, vp]
        _lib = lib
        return lib


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def _ptr(a):
    return a.ctypes.data_as(ctypes.c_void_p)


def nbox(L: int) -> int:
    """Number of boxes of a tree with L levels below the root: (4^(L+1) - 1) / 3."""
    return int(_load().orc_nbox(L))


def level_base(l: int) -> int:
    """Global id of the first box of level l (level order numbering)."""
    return (4 ** l - 1) // 3


class OracleError(RuntimeError):
    pass


def tree(x, y, L: int):
    """Median-split tree (Section 4).  Returns (perm[int32 N], rects[nbox,4] (x0,x1,y0,y1),
    leaf_begin[int64 4^L+1])."""
    x, y = _f64(x), _f64(y)
    n = x.shape[0]
    perm = np.empty(n, np.int32)
    rects = np.empty((nbox(L), 4), np.float64)
    lb = np.empty(4 ** L + 1, np.int64)
    rc = _load().orc_tree(n, _ptr(x), _ptr(y), L, _ptr(perm), _ptr(rects), _ptr(lb))
    if rc:
        raise OracleError(f"orc_tree failed ({rc})")
    return perm, rects, lb


def _root(root):
    return None if root is None else np.ascontiguousarray(root, np.float64)


def tree_uniform(x, y, L: int, root=None):
    """The uniform-grid mesh (square root, geometric quadrants) the adaptive one is compared with.
    ``root`` = (x0, y0, side) fixes the root square (default: the bounding square).  Returns
    (perm, rects, leaf_begin) like :func:`tree`; leaves may be empty."""
    x, y = _f64(x), _f64(y)
    n = x.shape[0]
    perm = np.empty(n, np.int32)
    rects = np.empty((nbox(L), 4), np.float64)
    lb = np.empty(4 ** L + 1, np.int64)
    r = _root(root)
    rc = _load().orc_tree_uniform(n, _ptr(x), _ptr(y), L, None if r is None else _ptr(r), _ptr(perm), _ptr(rects),
                                  _ptr(lb))
    if rc:
        raise OracleError(f"orc_tree_uniform failed ({rc})")
    return perm, rects, lb


def geometry(rects):
    """Centres (midpoints) and radii (half diagonals) of the boxes."""
    rects = _f64(rects)
    nb = rects.shape[0]
    c = np.empty((nb, 2), np.float64)
    r = np.empty(nb, np.float64)
    _load().orc_geometry(nb, _ptr(rects), _ptr(c), _ptr(r))
    return c, r


def theta_weak(c1, r1, c2, r2, theta) -> bool:
    """Criterion 2.1 for two spheres (disjointness included)."""
    return bool(_load().orc_theta_weak(float(c1[0]), float(c1[1]), float(r1),
                                       float(c2[0]), float(c2[1]), float(r2), float(theta)))


PARENT_FLAG = 0x40000000
SWAP_M2P = 0x20000000


def theta_swapped(c1, r1, c2, r2, theta) -> bool:
    """Criterion 2.1 with the roles of the two radii exchanged (disjointness included)."""
    return bool(_load().orc_theta_swapped(float(c1[0]), float(c1[1]), float(r1),
                                          float(c2[0]), float(c2[1]), float(r2), float(theta)))


def lists(rects, L: int, theta: float, parents: bool = False, swap: bool = False):
    """Connectivity of Section 4.  Returns (woff, widx, soff, sidx): CSR over all boxes in
    global id order; entries are within-level indices of the coupled boxes.  With ``parents``
    the optional optimisation of Section 4 is applied to the weak lists: four weak siblings whose
    parent satisfies the criterion become one entry (parent index | PARENT_FLAG).  With ``swap``
    the finest-level role exchange is applied too and (xoff, xidx) are appended: the leaf pairs
    taken out of the strong lists, SWAP_M2P marking those where the target is the larger leaf."""
    rects = _f64(rects)
    lib = _load()
    h = lib.orc_lists_build(L, _ptr(rects), float(theta))
    if parents:
        lib.orc_lists_merge_parents(h, _ptr(rects), float(theta))
    if swap:
        lib.orc_lists_swap_leaves(h, _ptr(rects), float(theta))
    try:
        out = []
        for kind in ((1, 0, 2) if swap else (1, 0)):
            tot = lib.orc_lists_total(h, kind)
            off = np.empty(nbox(L) + 1, np.int64)
            idx = np.empty(max(tot, 1), np.int32)
            lib.orc_lists_copy(h, kind, _ptr(off), _ptr(idx))
            out += [off, idx[:tot]]
    finally:
        lib.orc_lists_free(h)
    return tuple(out)


def _flags(parents, swap, uniform):
    return (1 if parents else 0) | (2 if swap else 0) | (4 if uniform else 0)


def fmm(x, y, q, L: int, p: int, theta: float, want_coeffs: bool = False, parents: bool = False,
        swap: bool = False, uniform: bool = False, root=None):
    """The whole method in FP64 (Section 4).  Returns phi in input order, plus the unscaled
    multipole and local coefficients (complex, [nbox, p+1]) when ``want_coeffs``.  ``parents``
    and ``swap`` apply the optional optimisations (see :func:`lists`); ``uniform`` runs the same
    method on the uniform-grid mesh (:func:`tree_uniform`), ``root`` = (x0, y0, side) on a given
    root square."""
    x, y, q = _f64(x), _f64(y), _f64(q)
    n = x.shape[0]
    phi = np.empty(n, np.float64)
    if root is not None:
        r = _root(root)
        rc = _load().orc_fmm_root(n, _ptr(x), _ptr(y), _ptr(q), L, p, float(theta), _flags(parents, swap, True),
                                  _ptr(r), _ptr(phi))
        if rc:
            raise OracleError(f"orc_fmm_root failed ({rc})")
        return phi
    if parents or swap or uniform:
        assert not want_coeffs
        flags = _flags(parents, swap, uniform)
        rc = _load().orc_fmm_ex(n, _ptr(x), _ptr(y), _ptr(q), L, p, float(theta), flags, _ptr(phi))
        if rc:
            raise OracleError(f"orc_fmm_ex failed ({rc})")
        return phi
    M = Lc = None
    mp = lp = None
    if want_coeffs:
        M = np.empty((nbox(L), p + 1), np.complex128)
        Lc = np.empty((nbox(L), p + 1), np.complex128)
        mp, lp = _ptr(M), _ptr(Lc)
    rc = _load().orc_fmm(n, _ptr(x), _ptr(y), _ptr(q), L, p, float(theta), _ptr(phi), mp, lp)
    if rc:
        raise OracleError(f"orc_fmm failed ({rc})")
    return (phi, M, Lc) if want_coeffs else phi


def direct(x, y, q, targets=None, nthreads: int = 0):
    """Eq. (1.1) by direct summation at the given input indices (all points by default)."""
    x, y, q = _f64(x), _f64(y), _f64(q)
    n = x.shape[0]
    t = np.arange(n, dtype=np.int64) if targets is None else np.ascontiguousarray(targets, np.int64)
    phi = np.empty(t.shape[0], np.float64)
    _load().orc_direct(n, _ptr(x), _ptr(y), _ptr(q), t.shape[0], _ptr(t), _ptr(phi), int(nthreads))
    return phi


def fmm_field(x, y, q, L: int, p: int, theta: float, parents: bool = False, swap: bool = False,
              uniform: bool = False):
    """The complex field F_i = sum_{j != i} -q_j / (z_i - z_j) by the method (Section 5's first
    experiment); returns a complex array in input order.  Options as :func:`fmm`."""
    x, y, q = _f64(x), _f64(y), _f64(q)
    n = x.shape[0]
    fre, fim = np.empty(n), np.empty(n)
    flags = _flags(parents, swap, uniform)
    rc = _load().orc_fmm_field_ex(n, _ptr(x), _ptr(y), _ptr(q), int(L), int(p), float(theta), flags,
                                  _ptr(fre), _ptr(fim))
    if rc:
        raise OracleError(f"orc_fmm_field returned {rc}")
    return fre + 1j * fim


def direct_field(x, y, q, targets=None, nthreads: int = 0):
    """The same field by direct summation at the given input indices (all points by default)."""
    x, y, q = _f64(x), _f64(y), _f64(q)
    n = x.shape[0]
    t = np.arange(n, dtype=np.int64) if targets is None else np.ascontiguousarray(targets, np.int64)
    fre, fim = np.empty(t.shape[0]), np.empty(t.shape[0])
    _load().orc_direct_field(n, _ptr(x), _ptr(y), _ptr(q), t.shape[0], _ptr(t), _ptr(fre), _ptr(fim), int(nthreads))
    return fre + 1j * fim


def _cvec(a, p):
    a = np.ascontiguousarray(a, np.complex128)
    assert a.shape[0] == p + 1
    return a


def p2m(x, y, q, center, p: int):
    """Multipole coefficients a_0..a_p about ``center`` (unscaled)."""
    x, y, q = _f64(x), _f64(y), _f64(q)
    a = np.empty(p + 1, np.complex128)
    _load().orc_p2m(x.shape[0], _ptr(x), _ptr(y), _ptr(q), float(center[0]), float(center[1]), p, _ptr(a))
    return a


def _op(name, c, z0, p):
    c = _cvec(c, p)
    out = np.empty(p + 1, np.complex128)
    getattr(_load(), name)(_ptr(c), float(np.real(z0)), float(np.imag(z0)), p, _ptr(out))
    return out


def m2m(a, z0, p: int):
    """Shift a multipole by z0 = c_child - c_parent."""
    return _op("orc_m2m", a, z0, p)


def m2l(a, z0, p: int):
    """Multipole about c_src to local about c_tgt, z0 = c_src - c_tgt."""
    return _op("orc_m2l", a, z0, p)


def l2l(b, z0, p: int):
    """Re-centre a local expansion, z0 = c_child - c_parent."""
    return _op("orc_l2l", b, z0, p)


def l2p(b, dz, p: int) -> float:
    """Re sum_l b_l dz^l."""
    b = _cvec(b, p)
    return float(_load().orc_l2p(_ptr(b), float(np.real(dz)), float(np.imag(dz)), p))


def p2l(x, y, q, center, p: int):
    """Local coefficients b_0..b_p about ``center`` of sources outside a disc about it (unscaled)."""
    x, y, q = _f64(x), _f64(y), _f64(q)
    b = np.empty(p + 1, np.complex128)
    _load().orc_p2l(x.shape[0], _ptr(x), _ptr(y), _ptr(q), float(center[0]), float(center[1]), p, _ptr(b))
    return b


def m2p(a, dz, p: int) -> float:
    """Re[a_0 log dz + sum_k a_k dz^-k]."""
    a = _cvec(a, p)
    return float(_load().orc_m2p(_ptr(a), float(np.real(dz)), float(np.imag(dz)), p))
