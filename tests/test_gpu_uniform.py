"""The uniform-grid mesh (the non-adaptive comparison of Section 5) on the GPU against the oracle:
the mesh (order, rectangles, leaf offsets) and the lists bit for bit, potentials and fields
within 1e-12 (binary64) and 1e-6 (mixed) -- with small leaves, with leaves of hundreds of
points, empty leaves and coincident points -- a forest, and a median build on the same handle
after a uniform one.
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


def _same_point(n=200):
    return W.Cloud(np.full(n, 0.25), np.full(n, -0.5), np.random.default_rng(3).normal(size=n), "same")


CASES = [
    ("normal_0.05", lambda: W.normal_sq(30000, 41, 0.05), 5),
    ("normal_0.003", lambda: W.normal_sq(20000, 42, 0.003), 5),
    ("layer_0.01", lambda: W.layer(30000, 43, 0.01), 6),
    ("uniform", lambda: W.uniform(4 ** 4 * 9 + 5, 44), 4),
    ("L1", lambda: W.normal_sq(300, 45, 0.1), 1),
    ("L0", lambda: W.uniform(50, 46), 0),
    ("same_point", _same_point, 2),
]


@pytest.fixture(scope="module")
def built(fmmlib, cuda):
    out = {}
    for name, make, L in CASES:
        c = make()
        out[name] = (c, L, fmmlib.FMM(_t(c.x, cuda), _t(c.y, cuda), L, 0.5, mesh="uniform"))
    yield out
    for _, _, f in out.values():
        f.close()


@pytest.mark.parametrize("name", [c[0] for c in CASES])
def test_mesh_and_lists_bit_exact(built, orc, name):
    c, L, f = built[name]
    perm, rects, lb = (a.cpu().numpy() for a in f.export_tree())
    op, orr, olb = orc.tree_uniform(c.x, c.y, L)
    assert np.array_equal(perm, op)
    assert np.array_equal(rects, orr)
    assert np.array_equal(lb.astype(np.int64), olb)
    woff, widx, soff, sidx = (a.cpu().numpy().astype(np.int64) for a in f.export_lists())
    ow, oi, os_, osi = orc.lists(orr, L, 0.5)
    assert np.array_equal(woff, ow) and np.array_equal(widx, oi)
    assert np.array_equal(soff, os_) and np.array_equal(sidx, osi)


@pytest.mark.parametrize("name", [c[0] for c in CASES])
@pytest.mark.parametrize("mode,p,tol", [("fp64", 17, 1e-12), ("mixed", 20, 1e-6)])
def test_potentials(built, orc, cuda, name, mode, p, tol):
    c, L, f = built[name]
    got = f.evaluate(_t(c.q, cuda), p, mode).cpu().numpy()
    ref = orc.fmm(c.x, c.y, c.q, L, p, 0.5, uniform=True)
    if name == "same_point":  # every pair coincides: all potentials are 0
        assert np.all(ref == 0) and np.max(np.abs(got)) == 0
        return
    assert relerr(got, ref) <= tol


def test_large_leaves_take_the_general_kernels(built, fmmlib):
    c, L, f = built["normal_0.003"]
    _, _, lb = (a.cpu().numpy() for a in f.export_tree())
    assert np.diff(lb).max() > 64  # the binary32 leaf-pair kernel covers leaves up to 64 points


@pytest.mark.parametrize("name", ["normal_0.05", "layer_0.01", "uniform"])
@pytest.mark.parametrize("mode,p,tol", [("fp64", 17, 1e-12), ("mixed", 20, 1e-6)])
def test_field(built, orc, cuda, name, mode, p, tol):
    c, L, f = built[name]
    got = f.evaluate_field(_t(c.q, cuda), p, mode).cpu().numpy()
    ref = orc.fmm_field(c.x, c.y, c.q, L, p, 0.5, uniform=True)
    assert relerr(got, ref) <= tol


def test_median_build_after_uniform(fmmlib, orc, cuda):
    c = W.layer(20000, 47, 0.02)
    L = 5
    x, y, q = _t(c.x, cuda), _t(c.y, cuda), _t(c.q, cuda)
    f = fmmlib.FMM(x, y, L, 0.5, mesh="uniform")
    try:
        ref_u = orc.fmm(c.x, c.y, c.q, L, 16, 0.5, uniform=True)
        assert relerr(f.evaluate(q, 16, "fp64").cpu().numpy(), ref_u) <= 1e-12
        f.mesh = "adaptive"
        f.rebuild(x, y)
        perm, rects, lb = (a.cpu().numpy() for a in f.export_tree())
        op, orr, olb = orc.tree(c.x, c.y, L)
        assert np.array_equal(perm, op) and np.array_equal(rects, orr) and np.array_equal(lb.astype(np.int64), olb)
        assert relerr(f.evaluate(q, 16, "fp64").cpu().numpy(), orc.fmm(c.x, c.y, c.q, L, 16, 0.5)) <= 1e-12
        assert relerr(f.evaluate(q, 20, "mixed").cpu().numpy(), orc.fmm(c.x, c.y, c.q, L, 20, 0.5)) <= 1e-6
        f.mesh = "uniform"
        f.rebuild(x, y)
        assert relerr(f.evaluate(q, 16, "fp64").cpu().numpy(), ref_u) <= 1e-12
    finally:
        f.close()


def test_uniform_forest(fmmlib, orc, cuda):
    clouds = [W.normal_sq(20000, 48, 0.01), W.uniform(3000, 49), W.layer(9000, 50, 0.005), W.uniform(40, 51)]
    levels = [5, 3, 5, 0]
    x = np.concatenate([c.x for c in clouds])
    y = np.concatenate([c.y for c in clouds])
    q = np.concatenate([c.q for c in clouds])
    b = fmmlib.FMMBatch(_t(x, cuda), _t(y, cuda), [c.x.shape[0] for c in clouds], levels, 0.5, mesh="uniform")
    try:
        for i, (c, L) in enumerate(zip(clouds, levels)):
            perm, rects, lb, woff, widx, soff, sidx = b.export_instance(i)
            op, orr, olb = orc.tree_uniform(c.x, c.y, L)
            assert np.array_equal(perm.cpu().numpy(), op)
            assert np.array_equal(rects.cpu().numpy(), orr)
            assert np.array_equal(lb.cpu().numpy().astype(np.int64), olb)
        for mode, p, tol in (("fp64", 16, 1e-12), ("mixed", 20, 1e-6)):
            phi = b.evaluate(_t(q, cuda), p, mode).cpu().numpy()
            for d, c, L in zip(b.inst, clouds, levels):
                ref = orc.fmm(c.x, c.y, c.q, L, p, 0.5, uniform=True)
                assert relerr(phi[d["p0"]:d["p0"] + d["n"]], ref) <= tol
    finally:
        b.close()


def test_uniform_with_section4_options(fmmlib, orc, cuda):
    c = W.normal_sq(30000, 52, 0.02)
    L = 5
    f = fmmlib.FMM(_t(c.x, cuda), _t(c.y, cuda), L, 0.5, mesh="uniform", parents=True, exchange=True)
    try:
        got = f.evaluate(_t(c.q, cuda), 17, "fp64").cpu().numpy()
        assert relerr(got, orc.fmm(c.x, c.y, c.q, L, 17, 0.5, parents=True, swap=True, uniform=True)) <= 1e-12
    finally:
        f.close()


@pytest.mark.parametrize("mesh", ["adaptive", "uniform"])
def test_collapsed_leaf_pairs(fmmlib, cuda, mesh):
    # every point at one place: leaf pairs of zero extent; all potentials are 0 in both paths
    c = _same_point(256)
    f = fmmlib.FMM(_t(c.x, cuda), _t(c.y, cuda), 2, 0.5, mesh=mesh)
    try:
        for mode in ("mixed", "fp64"):
            got = f.evaluate(_t(c.q, cuda), 20, mode).cpu().numpy()
            assert np.max(np.abs(got)) == 0
    finally:
        f.close()


@pytest.mark.parametrize("root", [(0.0, 0.0, 1.0), (-0.25, -0.5, 2.0)])
def test_fixed_root_square(fmmlib, orc, cuda, root):
    c = W.normal_sq(30000, 53, 0.01)
    L = 6
    f = fmmlib.FMM(_t(c.x, cuda), _t(c.y, cuda), L, 0.5, mesh="uniform", root=root)
    try:
        perm, rects, lb = (a.cpu().numpy() for a in f.export_tree())
        op, orr, olb = orc.tree_uniform(c.x, c.y, L, root=root)
        assert np.array_equal(perm, op) and np.array_equal(rects, orr)
        assert np.array_equal(lb.astype(np.int64), olb)
        for mode, p, tol in (("fp64", 16, 1e-12), ("mixed", 20, 1e-6)):
            got = f.evaluate(_t(c.q, cuda), p, mode).cpu().numpy()
            assert relerr(got, orc.fmm(c.x, c.y, c.q, L, p, 0.5, root=root)) <= tol
    finally:
        f.close()


def test_one_giant_leaf_mixed(fmmlib, orc, cuda):
    # a tight cluster in the unit-square mesh: nearly every point in one leaf, which the general
    # near-field kernel spreads over many warps; the mixed path stays within 1e-6 of the direct sum
    c = W.normal_sq(60000, 54, 0.002)
    L = 5
    f = fmmlib.FMM(_t(c.x, cuda), _t(c.y, cuda), L, 0.5, mesh="uniform", root=(0.0, 0.0, 1.0))
    try:
        lb = f.export_tree()[2].cpu().numpy()
        assert np.diff(lb).max() > 50000
        tg = W.sample_targets(c.x.size, 1000, 55)
        ref = orc.direct(c.x, c.y, c.q, tg, nthreads=0)
        got = f.evaluate(_t(c.q, cuda), 20, "mixed").cpu().numpy()[tg]
        assert relerr(got, ref) <= 1e-6
        got = f.evaluate(_t(c.q, cuda), 20, "fp64").cpu().numpy()[tg]
        assert relerr(got, ref) <= 1e-10
    finally:
        f.close()
