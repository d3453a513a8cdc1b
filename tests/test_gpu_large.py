"""The large nonuniform workload at full size: N = 2^24 points, 80% on 20 rings (radial spread
1e-3) and 20% in a Plummer-like core, strengths uniform in [0, 1], 9 levels (64 points per leaf),
theta = 1/2, p = 30, tolerance 1e-10.

A tolerance below 1e-7 runs the binary64 path (the mixed path's binary32 expansions cannot reach
it), so the check is against the oracle's binary64 direct sum on 2,048 sampled targets.  The
tree is checked through properties that hold at any size (the oracle's full-size tree would take
minutes): the permutation, the balanced leaf sizes, and every point inside its leaf rectangle.
"""
import numpy as np
import pytest

from paper_1006_2269_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def _t(a, dev):
    import torch
    return torch.as_tensor(np.ascontiguousarray(a), device=dev)


def relerr(a, ref):
    return float(np.max(np.abs(a - ref)) / np.max(np.abs(ref)))


@pytest.fixture(scope="module")
def large(fmmlib, cuda):
    w = W.LARGE_16M
    c = W.large_16m_cloud()
    f = fmmlib.FMM(_t(c.x, cuda), _t(c.y, cuda), w.levels, w.theta)
    yield w, c, f
    f.close()


def test_large_tree_properties(large):
    w, c, f = large
    perm, rects, lb = (a.cpu().numpy() for a in f.export_tree())
    n, L = w.n, w.levels
    assert np.array_equal(np.sort(perm), np.arange(n))
    sizes = np.diff(lb.astype(np.int64))
    assert sizes.min() >= n // 4 ** L and sizes.max() <= -(-n // 4 ** L)
    leaf = np.repeat(np.arange(4 ** L), sizes)
    r = rects[(4 ** L - 1) // 3 + leaf]
    x, y = c.x[perm], c.y[perm]
    assert np.all((r[:, 0] <= x) & (x <= r[:, 1]) & (r[:, 2] <= y) & (y <= r[:, 3]))


def test_large_tolerance_1e10_vs_direct(large, orc, cuda):
    w, c, f = large
    tg = W.sample_targets(w.n, w.n_check, W.SEED_BASE + 4 + 100)
    ref = orc.direct(c.x, c.y, c.q, tg, nthreads=0)
    phi = f.evaluate(_t(c.q, cuda), w.p, "mixed", tol=1e-10).cpu().numpy()[tg]
    assert relerr(phi, ref) <= 1e-10
    # the split mode (binary64 expansions, float-float near field) at the same tolerance
    phi = f.evaluate(_t(c.q, cuda), w.p, "split", tol=1e-10).cpu().numpy()[tg]
    assert relerr(phi, ref) <= 1e-10
    # the mixed path at its own tolerance on the same input
    phi = f.evaluate(_t(c.q, cuda), 20, "mixed", tol=1e-6).cpu().numpy()[tg]
    assert relerr(phi, ref) <= 1e-6
