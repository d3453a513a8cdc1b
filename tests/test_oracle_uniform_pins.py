"""Pins of the oracle's uniform-grid mesh (the non-adaptive comparison of Section 5), on the CPU.

Geometry: the root is a square on the bounding box's lower-left corner, children are the four
exact quadrants of their parent, and the leaves are congruent squares tiling the root.  Points:
every point lies in its leaf square, and the leaf counts equal numpy's 2-D histogram over the
same grid.  On a symmetric lattice the uniform grid and the median splits put the same points in
the same leaves (their rectangles differ).  The method on the uniform mesh equals the direct sum
when there is no far field and converges in p like the adaptive one.
"""
import numpy as np
import pytest

import oracle
from paper_1006_2269_gb300 import workloads as W


def _base(l):
    return (4 ** l - 1) // 3


@pytest.mark.parametrize("L", [0, 1, 3, 5])
def test_quadrants_tile_the_root_square(L):
    c = W.layer(5000, 11, 0.03)
    _, rects, _ = oracle.tree_uniform(c.x, c.y, L)
    r0 = rects[0]
    side = max(c.x.max() - c.x.min(), c.y.max() - c.y.min())
    assert r0[0] == c.x.min() and r0[2] == c.y.min()
    assert np.isclose(r0[1] - r0[0], side, rtol=1e-15) and np.isclose(r0[3] - r0[2], side, rtol=1e-15)
    for l in range(L):
        for b in range(4 ** l):
            p = rects[_base(l) + b]
            ch = rects[_base(l + 1) + 4 * b:_base(l + 1) + 4 * b + 4]
            xm, ym = ch[0, 1], ch[0, 3]
            assert np.isclose(xm, 0.5 * (p[0] + p[1]), rtol=0, atol=1e-15) and np.isclose(ym, 0.5 * (p[2] + p[3]), rtol=0, atol=1e-15)
            # (x-low, y-low), (x-low, y-high), (x-high, y-low), (x-high, y-high)
            assert np.array_equal(ch[:, 0], [p[0], p[0], xm, xm]) and np.array_equal(ch[:, 1], [xm, xm, p[1], p[1]])
            assert np.array_equal(ch[:, 2], [p[2], ym, p[2], ym]) and np.array_equal(ch[:, 3], [ym, p[3], ym, p[3]])
    leaves = rects[_base(L):_base(L) + 4 ** L]
    assert np.allclose(leaves[:, 1] - leaves[:, 0], side / 2 ** L, rtol=1e-12)
    assert np.allclose(leaves[:, 3] - leaves[:, 2], side / 2 ** L, rtol=1e-12)


@pytest.mark.parametrize("make,L", [(lambda: W.normal_sq(20000, 12, 0.02), 5), (lambda: W.uniform(7000, 13), 4),
                                    (lambda: W.layer(9000, 14, 0.005), 6)])
def test_points_in_leaves_and_counts(make, L):
    c = make()
    perm, rects, lb = oracle.tree_uniform(c.x, c.y, L)
    assert np.array_equal(np.sort(perm), np.arange(c.x.size))
    leaf = np.repeat(np.arange(4 ** L), np.diff(lb))
    r = rects[_base(L) + leaf]
    x, y = c.x[perm], c.y[perm]
    tol = 1e-12 * (rects[0, 1] - rects[0, 0])
    assert np.all((r[:, 0] - tol <= x) & (x <= r[:, 1] + tol) & (r[:, 2] - tol <= y) & (y <= r[:, 3] + tol))
    # inside a leaf: ascending input index
    for b in range(4 ** L):
        seg = perm[lb[b]:lb[b + 1]]
        assert np.all(np.diff(seg) > 0)
    # counts against numpy's histogram over the same grid, cell (ix, iy) -> leaf id by digits
    m = 2 ** L
    edges_x = np.linspace(rects[0, 0], rects[0, 1], m + 1)
    edges_y = np.linspace(rects[0, 2], rects[0, 3], m + 1)
    H, _, _ = np.histogram2d(c.x, c.y, bins=[edges_x, edges_y])
    ids = np.zeros((m, m), np.int64)
    for ix in range(m):
        for iy in range(m):
            v = 0
            for j in range(L - 1, -1, -1):
                v = 4 * v + 2 * ((ix >> j) & 1) + ((iy >> j) & 1)
            ids[ix, iy] = v
    counts = np.zeros(4 ** L, np.int64)
    counts[ids.ravel()] = H.ravel().astype(np.int64)
    assert np.array_equal(np.diff(lb), counts)


def test_lattice_matches_the_median_tree():
    g = np.arange(64) + 0.5
    X, Y = np.meshgrid(g, g, indexing="ij")
    x, y = X.ravel() / 64, Y.ravel() / 64
    for L in (1, 2, 3, 4):
        pu, ru, lu = oracle.tree_uniform(x, y, L)
        pm, rm, lm = oracle.tree(x, y, L)
        assert np.array_equal(pu, pm) and np.array_equal(lu, lm)
        if L >= 2:
            assert not np.array_equal(ru, rm)


def test_clustered_leaves_are_unbalanced():
    c = W.normal_sq(50000, 15, 0.01)
    _, _, lb = oracle.tree_uniform(c.x, c.y, 5)
    sizes = np.diff(lb)
    assert sizes.max() > 10 * (50000 / 4 ** 5) and np.sum(sizes == 0) > 0


def test_all_points_equal():
    x = np.full(100, 0.3)
    y = np.full(100, -0.7)
    perm, rects, lb = oracle.tree_uniform(x, y, 2)
    assert np.array_equal(perm, np.arange(100)) and lb[1] == 100 and lb[-1] == 100
    assert np.all(rects[:, 0] == 0.3) and np.all(rects[:, 1] == 0.3)


@pytest.mark.parametrize("L", [0, 1])
def test_method_without_far_field_is_direct(L):
    c = W.normal_sq(900, 16, 0.1)
    f = oracle.fmm(c.x, c.y, c.q, L, 10, 0.5, uniform=True)
    d = oracle.direct(c.x, c.y, c.q)
    assert np.max(np.abs(f - d)) <= 1e-13 * np.max(np.abs(d))


@pytest.mark.parametrize("make", [lambda: W.normal_sq(8000, 17, 0.05), lambda: W.layer(8000, 18, 0.01)])
def test_method_converges(make):
    c = make()
    d = oracle.direct(c.x, c.y, c.q)
    errs = []
    for p in (4, 8, 12, 16):
        f = oracle.fmm(c.x, c.y, c.q, 5, p, 0.5, uniform=True)
        errs.append(np.max(np.abs(f - d)) / np.max(np.abs(d)))
    errs = np.array(errs)
    assert np.all(errs[1:] <= errs[:-1] / 8)
    assert np.all(errs <= 0.5 ** (np.array([4, 8, 12, 16]) + 1) / 0.25)
    fe = oracle.fmm_field(c.x, c.y, c.q, 5, 16, 0.5, uniform=True)
    de = oracle.direct_field(c.x, c.y, c.q)
    assert np.max(np.abs(fe - de)) / np.max(np.abs(de)) <= 0.5 ** 17 / 0.25


def test_fixed_unit_square_root():
    # Section 5's experiment puts every point in the unit square; with that square as the root
    # the leaves are the dyadic squares [i/2^L, (i+1)/2^L] x [j/2^L, (j+1)/2^L] exactly
    c = W.normal_sq(6000, 19, 0.05)
    L = 4
    perm, rects, lb = oracle.tree_uniform(c.x, c.y, L, root=(0.0, 0.0, 1.0))
    m = 2 ** L
    leaves = rects[_base(L):]
    assert np.all(np.isin(leaves[:, 0] * m, np.arange(m))) and np.all(leaves[:, 1] - leaves[:, 0] == 1.0 / m)
    H, _, _ = np.histogram2d(c.x, c.y, bins=[np.linspace(0, 1, m + 1), np.linspace(0, 1, m + 1)])
    assert np.diff(lb).max() == H.max() and np.sum(np.diff(lb) > 0) == np.sum(H > 0)
    d = oracle.direct(c.x, c.y, c.q)
    errs = [np.max(np.abs(oracle.fmm(c.x, c.y, c.q, L, p, 0.5, root=(0.0, 0.0, 1.0)) - d)) / np.max(np.abs(d))
            for p in (6, 12)]
    assert errs[1] <= errs[0] / 8 and errs[1] <= 0.5 ** 13 / 0.25
