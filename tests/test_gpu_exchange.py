"""The finest-level role exchange (Section 4's second structural optimisation) on the GPU against
the oracle in the same mode: the weak, strong and exchange lists bit for bit (with and without
parent-level entries), potentials and fields within 1e-12 (binary64) and 1e-6 (mixed, both M2L
kernels), a forest, mode switches on one lists object, the capacity regrowth when the exchange
lists overflow, and the full-size clustered workload against the direct sum at sampled targets.
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


CASES = [
    ("clusters", lambda: W.clusters(30011, 81), 5),
    ("rings", lambda: W.rings_plummer(40000, 82), 6),
    ("circle", lambda: W.circle(20000, 83), 5),
    ("uniform_ragged", lambda: W.uniform(4 ** 4 * 5 + 77, 84), 4),
    ("L1", lambda: W.uniform(101, 85), 1),
    ("big_leaves", lambda: W.normal(4 ** 3 * 90, 86), 3),  # 90 points per leaf: binary64 near field
]


@pytest.fixture(scope="module")
def built(fmmlib, cuda):
    out = {}
    for name, make, L in CASES:
        c = make()
        out[name] = (c, L, fmmlib.FMM(_t(c.x, cuda), _t(c.y, cuda), L, 0.5, exchange=True))
    yield out
    for _, _, f in out.values():
        f.close()


def _check_lists(f, orc, c, L, theta, parents):
    woff, widx, soff, sidx = (a.cpu().numpy().astype(np.int64) for a in f.export_lists())
    xoff, xidx = (a.cpu().numpy().astype(np.int64) for a in f.export_exchange())
    _, rects, _ = orc.tree(c.x, c.y, L)
    ow, oi, os_, osi, ox, oxi = orc.lists(rects, L, theta, parents=parents, swap=True)
    assert np.array_equal(woff, ow) and np.array_equal(widx, oi)
    assert np.array_equal(soff, os_) and np.array_equal(sidx, osi)
    assert np.array_equal(xoff, ox) and np.array_equal(xidx, oxi)
    return int(ox[-1])


@pytest.mark.parametrize("theta", [0.5, 0.3])
@pytest.mark.parametrize("name", [c[0] for c in CASES])
def test_exchange_lists_bit_exact(built, orc, cuda, name, theta):
    c, L, f = built[name]
    if theta != 0.5:
        f.rebuild(_t(c.x, cuda), _t(c.y, cuda), theta=theta)
    try:
        nx = _check_lists(f, orc, c, L, theta, parents=False)
        if name in ("clusters", "rings", "circle"):
            assert nx > 0
    finally:
        if theta != 0.5:
            f.rebuild(_t(c.x, cuda), _t(c.y, cuda), theta=0.5)


@pytest.mark.parametrize("name", [c[0] for c in CASES])
@pytest.mark.parametrize("mode,p,tol,kind", [("fp64", 17, 1e-12, 0), ("mixed", 20, 1e-6, 1), ("mixed", 20, 1e-6, 2),
                                             ("mixed", 30, 1e-6, 0), ("split", 17, 1e-11, 0),
                                             ("split", 30, 1e-11, 0)])
def test_exchange_potentials(built, orc, fmmlib, cuda, name, mode, p, tol, kind):
    c, L, f = built[name]
    fmmlib.fmm_set_m2l_kernel(f.tree, kind)
    try:
        got = f.evaluate(_t(c.q, cuda), p, mode).cpu().numpy()
    finally:
        fmmlib.fmm_set_m2l_kernel(f.tree, 0)
    ref = orc.fmm(c.x, c.y, c.q, L, p, 0.5, swap=True)
    assert relerr(got, ref) <= tol


@pytest.mark.parametrize("name", ["clusters", "rings", "circle", "uniform_ragged"])
@pytest.mark.parametrize("mode,p,tol", [("fp64", 17, 1e-12), ("mixed", 20, 1e-6)])
def test_exchange_field(built, orc, cuda, name, mode, p, tol):
    c, L, f = built[name]
    got = f.evaluate_field(_t(c.q, cuda), p, mode).cpu().numpy()
    ref = orc.fmm_field(c.x, c.y, c.q, L, p, 0.5, swap=True)
    assert relerr(got, ref) <= tol


@pytest.mark.parametrize("n,L,seed", [(4 ** 3 * 200, 3, 93), (4 ** 2 * 700 + 9, 2, 94)])
def test_exchange_split_large_leaves(fmmlib, orc, cuda, n, L, seed):
    # leaves of 200 and about 700 points: the float-float M2P's lanes hold more than their four
    # points in registers and take the rest one at a time
    c = W.normal(n, seed)
    f = fmmlib.FMM(_t(c.x, cuda), _t(c.y, cuda), L, 0.5, exchange=True)
    try:
        assert _check_lists(f, orc, c, L, 0.5, parents=False) > 0
        got = f.evaluate(_t(c.q, cuda), 20, "split").cpu().numpy()
    finally:
        f.close()
    assert relerr(got, orc.fmm(c.x, c.y, c.q, L, 20, 0.5, swap=True)) <= 1e-11


def test_exchange_with_parent_entries(fmmlib, orc, cuda):
    c = W.clusters(25000, 87)
    L = 5
    f = fmmlib.FMM(_t(c.x, cuda), _t(c.y, cuda), L, 0.5, parents=True, exchange=True)
    try:
        assert _check_lists(f, orc, c, L, 0.5, parents=True) > 0
        for mode, p, tol in (("fp64", 17, 1e-12), ("mixed", 20, 1e-6), ("split", 24, 1e-11)):
            got = f.evaluate(_t(c.q, cuda), p, mode).cpu().numpy()
            assert relerr(got, orc.fmm(c.x, c.y, c.q, L, p, 0.5, parents=True, swap=True)) <= tol
    finally:
        f.close()


def test_exchange_forest(fmmlib, orc, cuda):
    clouds = [W.clusters(20000, 88), W.uniform(5000, 89), W.uniform(40, 90), W.circle(9000, 91)]
    levels = [5, 4, 0, 5]
    x = np.concatenate([c.x for c in clouds])
    y = np.concatenate([c.y for c in clouds])
    q = np.concatenate([c.q for c in clouds])
    b = fmmlib.FMMBatch(_t(x, cuda), _t(y, cuda), [c.x.shape[0] for c in clouds], levels, 0.5, exchange=True)
    try:
        for i, (c, L) in enumerate(zip(clouds, levels)):
            _, rects, _, woff, widx, soff, sidx = b.export_instance(i)
            xoff, xidx = b.export_exchange(i)
            ow, oi, os_, osi, ox, oxi = orc.lists(rects.cpu().numpy(), L, 0.5, swap=True)
            assert np.array_equal(soff.cpu().numpy().astype(np.int64), os_)
            assert np.array_equal(sidx.cpu().numpy().astype(np.int64), osi)
            assert np.array_equal(xoff.cpu().numpy().astype(np.int64), ox)
            assert np.array_equal(xidx.cpu().numpy().astype(np.int64), oxi)
        for mode, p, tol in (("fp64", 16, 1e-12), ("mixed", 20, 1e-6), ("split", 20, 1e-11)):
            phi = b.evaluate(_t(q, cuda), p, mode).cpu().numpy()
            for d, c, L in zip(b.inst, clouds, levels):
                ref = orc.fmm(c.x, c.y, c.q, L, p, 0.5, swap=True)
                assert relerr(phi[d["p0"]:d["p0"] + d["n"]], ref) <= tol
    finally:
        b.close()


def test_mode_switches(fmmlib, orc, cuda):
    c = W.rings_plummer(30000, 92)
    L = 5
    f = fmmlib.FMM(_t(c.x, cuda), _t(c.y, cuda), L, 0.5)
    try:
        _, rects, _ = orc.tree(c.x, c.y, L)
        for mode in (2, 0, 3, 1, 2):
            fmmlib.fmm_lists_set_mode(f.lists, mode)
            fmmlib.fmm_interaction_lists(f.tree, f.lists, 0.5)
            woff, widx, soff, sidx = (a.cpu().numpy().astype(np.int64) for a in f.export_lists())
            ref = orc.lists(rects, L, 0.5, parents=bool(mode & 1), swap=bool(mode & 2))
            assert np.array_equal(woff, ref[0]) and np.array_equal(widx, ref[1])
            assert np.array_equal(soff, ref[2]) and np.array_equal(sidx, ref[3])
            if mode & 2:
                xoff, xidx = (a.cpu().numpy().astype(np.int64) for a in f.export_exchange())
                assert np.array_equal(xoff, ref[4]) and np.array_equal(xidx, ref[5])
            got = f.evaluate(_t(c.q, cuda), 16, "fp64").cpu().numpy()
            assert relerr(got, orc.fmm(c.x, c.y, c.q, L, 16, 0.5, parents=bool(mode & 1), swap=bool(mode & 2))) <= 1e-12
    finally:
        f.close()


def test_exchange_capacity_regrowth(fmmlib, orc, cuda):
    # a strong capacity far below the exchange count: the first build overflows, the class
    # regrows from the exchange count and the rebuilt lists match the oracle
    c = W.clusters(20000, 93)
    L = 5
    f = fmmlib.FMM(_t(c.x, cuda), _t(c.y, cuda), L, 0.5, weak_capacity=200000, strong_capacity=300,
                   exchange=True)
    try:
        assert _check_lists(f, orc, c, L, 0.5, parents=False) > 300
        got = f.evaluate(_t(c.q, cuda), 17, "fp64").cpu().numpy()
        assert relerr(got, orc.fmm(c.x, c.y, c.q, L, 17, 0.5, swap=True)) <= 1e-12
    finally:
        f.close()


def test_full_size_clusters_vs_direct(fmmlib, orc, cuda):
    # 2^20 clustered points, 8 levels, p = 20: mixed within 1e-6 of the direct sum on 2,048
    # sampled targets, with and without parent-level entries
    import torch
    w = W.MIXED_1M
    c = W.mixed_1m_cloud()
    tg = W.sample_targets(w.n, 2048, W.SEED_BASE + 130)
    ref = orc.direct(c.x, c.y, c.q, tg, nthreads=0)
    x, y, q = _t(c.x, cuda), _t(c.y, cuda), _t(c.q, cuda)
    for parents in (False, True):
        f = fmmlib.FMM(x, y, w.levels, w.theta, parents=parents, exchange=True)
        try:
            phi = f.evaluate(q, w.p, "mixed").cpu().numpy()[tg]
            assert relerr(phi, ref) <= 1e-6
            nx = fmmlib.fmm_lists_export_exchange(f.lists, 0)
            assert nx > 0
        finally:
            f.close()
    torch.cuda.synchronize()
