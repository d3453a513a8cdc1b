"""Batched evaluation: a forest of independent instances in one set of launches.

Every instance of a forest must give exactly what the oracle gives for that point set alone:
tree and lists bit for bit, binary64 potentials within 1e-12, mixed within 1e-6.  The full-size
batched workload (512 instances, N log-uniform in [1e3, 2e5], uniform / normal / jittered circle,
leaves of ~32 points, theta = 1/2, p = 16) is checked against the oracle FMM on a sample of
instances and against the direct sum on sampled targets of every instance.
"""
import numpy as np
import pytest

from paper_1006_2269_gb300 import workloads as W

pytestmark = pytest.mark.gpu

TOL_FP64 = 1e-12
TOL_MIXED = 1e-6


def _t(a, dev):
    import torch
    return torch.as_tensor(np.ascontiguousarray(a), device=dev)


def relerr(a, ref):
    return float(np.max(np.abs(a - ref)) / np.max(np.abs(ref)))


def _collinear(n, seed):
    c = W.uniform(n, seed)
    return W.Cloud(c.x, np.full(n, 0.75), c.q, "collinear")


def _dupes(n, seed):
    c = W.uniform(n, seed)
    return W.Cloud(np.round(c.x * 8) / 8, np.round(c.y * 8) / 8, c.q, "dupes")


# (cloud, levels): uneven sizes, every level count from 0 to 5, ragged and exact 4^L sizes,
# degenerate geometry, an instance of one tile and one spanning several
SMALL_FOREST = [
    (lambda: W.uniform(37, 101), 0),
    (lambda: W.clusters(9000, 102), 4),
    (lambda: W.uniform(101, 103), 1),
    (lambda: W.uniform(4 ** 3 + 13, 104), 3),
    (lambda: W.circle(5000, 105), 4),
    (lambda: W.normal(1234, 106), 2),
    (lambda: W.uniform(4 ** 4, 107), 4),
    (lambda: _collinear(2000, 108), 3),
    (lambda: _dupes(1500, 109), 2),
    (lambda: W.rings_plummer(20000, 110), 5),
    (lambda: W.uniform(3, 111), 0),
]


def _concat(clouds):
    x = np.concatenate([c.x for c in clouds])
    y = np.concatenate([c.y for c in clouds])
    q = np.concatenate([c.q for c in clouds])
    return x, y, q


@pytest.fixture(scope="module")
def forest(fmmlib, cuda):
    clouds = [make() for make, _ in SMALL_FOREST]
    levels = [L for _, L in SMALL_FOREST]
    x, y, q = _concat(clouds)
    b = fmmlib.FMMBatch(_t(x, cuda), _t(y, cuda), [c.x.shape[0] for c in clouds], levels, 0.5)
    yield clouds, levels, (x, y, q), b
    b.close()


def _slices(b):
    return [(d["p0"], d["p0"] + d["n"]) for d in b.inst]


def test_instance_table(forest, fmmlib):
    clouds, levels, _, b = forest
    assert fmmlib.fmm_tree_num_instances(b.tree) == len(clouds)
    p0 = b0 = lb0 = 0
    for c, L, d in zip(clouds, levels, b.inst):
        n = c.x.shape[0]
        assert (d["p0"], d["n"], d["levels"], d["b0"], d["lb0"]) == (p0, n, L, b0, lb0)
        assert d["nbox"] == (4 ** (L + 1) - 1) // 3
        p0 += n
        b0 += d["nbox"]
        lb0 += 4 ** L + 1


@pytest.mark.parametrize("i", range(len(SMALL_FOREST)))
def test_forest_tree_and_lists_bit_exact(forest, orc, i):
    clouds, levels, _, b = forest
    c, L = clouds[i], levels[i]
    perm, rects, lb, woff, widx, soff, sidx = b.export_instance(i)
    operm, orects, olb = orc.tree(c.x, c.y, L)
    assert np.array_equal(perm.cpu().numpy(), operm)
    assert np.array_equal(lb.cpu().numpy().astype(np.int64), olb)
    assert np.array_equal(rects.cpu().numpy(), orects)
    owoff, owidx, osoff, osidx = orc.lists(orects, L, 0.5)
    assert np.array_equal(woff.cpu().numpy().astype(np.int64), owoff)
    assert np.array_equal(soff.cpu().numpy().astype(np.int64), osoff)
    assert np.array_equal(widx.cpu().numpy().astype(np.int64), owidx)
    assert np.array_equal(sidx.cpu().numpy().astype(np.int64), osidx)


@pytest.mark.parametrize("mode,p,tol", [("fp64", 17, TOL_FP64), ("fp64", 6, TOL_FP64),
                                        ("mixed", 16, TOL_MIXED), ("mixed", 20, TOL_MIXED)])
def test_forest_potentials(forest, orc, cuda, mode, p, tol):
    clouds, levels, (x, y, q), b = forest
    phi = b.evaluate(_t(q, cuda), p, mode).cpu().numpy()
    for (a, e), c, L in zip(_slices(b), clouds, levels):
        ref = orc.fmm(c.x, c.y, c.q, L, p, 0.5)
        assert relerr(phi[a:e], ref) <= tol, (c.name, L)


def test_forest_tight_tolerance_takes_split(forest, orc, cuda):
    # a requested tolerance below what binary32 expansions reach runs the split precision
    # (binary64 expansions, float-float near field), accurate to the binary64 bound
    clouds, levels, (x, y, q), b = forest
    phi = b.evaluate(_t(q, cuda), 24, "mixed", tol=1e-10).cpu().numpy()
    for (a, e), c, L in zip(_slices(b), clouds, levels):
        ref = orc.fmm(c.x, c.y, c.q, L, 24, 0.5)
        assert relerr(phi[a:e], ref) <= TOL_FP64


def test_forest_theta_rebuild(forest, orc, cuda):
    clouds, levels, (x, y, q), b = forest
    b.rebuild(_t(x, cuda), _t(y, cuda), theta=0.3)
    try:
        for i, (c, L) in enumerate(zip(clouds, levels)):
            _, rects, _, woff, widx, soff, sidx = b.export_instance(i)
            owoff, owidx, osoff, osidx = orc.lists(rects.cpu().numpy(), L, 0.3)
            assert np.array_equal(woff.cpu().numpy().astype(np.int64), owoff)
            assert np.array_equal(widx.cpu().numpy().astype(np.int64), owidx)
            assert np.array_equal(soff.cpu().numpy().astype(np.int64), osoff)
            assert np.array_equal(sidx.cpu().numpy().astype(np.int64), osidx)
    finally:
        b.rebuild(_t(x, cuda), _t(y, cuda), theta=0.5)


def test_forest_capacity_regrow(fmmlib, orc, cuda):
    # deliberately small per-instance capacities: the overflow is reported per instance and the
    # class regrows exactly the instances that need it
    clouds = [W.clusters(6000, 120), W.uniform(500, 121)]
    levels = [4, 2]
    x, y, q = _concat(clouds)
    tree = fmmlib.fmm_tree_create_batched([6000, 500], levels)
    try:
        nb = [fmmlib.fmm_tree_instance(tree, i)["nbox"] for i in range(2)]
        lists = fmmlib.fmm_lists_create_batched(tree, [16, 10 * nb[1]], [16, 10 * nb[1]])
        try:
            fmmlib.fmm_build_tree(tree, _t(x, cuda), _t(y, cuda))
            fmmlib.fmm_interaction_lists(tree, lists, 0.5)
            w, s, over = fmmlib.fmm_lists_counts(lists, 2, check=False)
            assert over
            _, orects0, _ = orc.tree(clouds[0].x, clouds[0].y, 4)
            ow0, _, os0, _ = orc.lists(orects0, 4, 0.5)
            _, orects1, _ = orc.tree(clouds[1].x, clouds[1].y, 2)
            ow1, _, os1, _ = orc.lists(orects1, 2, 0.5)
            assert w[0] <= ow0[-1] and s[0] <= os0[-1]  # lower bounds for the instance that overflowed
            assert (w[1], s[1]) == (ow1[-1], os1[-1])    # exact for the one that fit
            with pytest.raises(fmmlib.FMMError) as ei:
                fmmlib.fmm_lists_sync(lists)
            assert ei.value.code == fmmlib.FMM_ERR_CAPACITY
            with pytest.raises(fmmlib.FMMError) as ei:
                fmmlib.fmm_sync_status(tree, lists)
            assert ei.value.code == fmmlib.FMM_ERR_CAPACITY
        finally:
            fmmlib.fmm_lists_destroy(lists)
    finally:
        fmmlib.fmm_tree_destroy(tree)
    # the class grows the capacities until the lists fit
    b = fmmlib.FMMBatch(_t(x, cuda), _t(y, cuda), [6000, 500], levels, 0.5, weak_per_box=1, strong_per_box=1)
    try:
        phi = b.evaluate(_t(q, cuda), 12, "fp64").cpu().numpy()
        assert relerr(phi[:6000], orc.fmm(clouds[0].x, clouds[0].y, clouds[0].q, 4, 12, 0.5)) <= TOL_FP64
        assert relerr(phi[6000:], orc.fmm(clouds[1].x, clouds[1].y, clouds[1].q, 2, 12, 0.5)) <= TOL_FP64
    finally:
        b.close()


def test_forest_graph_replay_and_autotune(forest, orc, cuda, fmmlib):
    import torch
    clouds, levels, (x, y, q), b = forest
    qd = _t(q, cuda)
    m2l, p2p = b.autotune(qd, 16)
    assert m2l >= 1 and p2p >= 1
    out = torch.empty(b.n, dtype=torch.float64, device=cuda)
    xd, yd = _t(x, cuda), _t(y, cuda)
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(s):  # warm-up outside capture (workspace allocation)
        fmmlib.fmm_build_tree(b.tree, xd, yd)
        fmmlib.fmm_interaction_lists(b.tree, b.lists, 0.5)
        fmmlib.fmm_evaluate(b.tree, b.lists, qd, 16, fmmlib.FMM_MODE_MIXED, out)
    torch.cuda.current_stream().wait_stream(s)
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        fmmlib.fmm_build_tree(b.tree, xd, yd)
        fmmlib.fmm_interaction_lists(b.tree, b.lists, 0.5)
        fmmlib.fmm_evaluate(b.tree, b.lists, qd, 16, fmmlib.FMM_MODE_MIXED, out)
    out.zero_()
    g.replay()
    torch.cuda.synchronize()
    fmmlib.fmm_sync_status(b.tree, b.lists)
    phi = out.cpu().numpy()
    for (a, e), c, L in zip(_slices(b), clouds, levels):
        ref = orc.fmm(c.x, c.y, c.q, L, 16, 0.5)
        assert relerr(phi[a:e], ref) <= TOL_MIXED
    fmmlib.fmm_set_launch(b.tree, 0, 0)


def test_forest_create_errors(fmmlib, cuda):
    with pytest.raises(fmmlib.FMMError) as ei:
        fmmlib.fmm_tree_create_batched([100, 10], [2, 2])  # 10 < 4^2
    assert ei.value.code == fmmlib.FMM_ERR_LEVELS
    with pytest.raises(fmmlib.FMMError) as ei:
        fmmlib.fmm_tree_create_batched([100, 0], [1, 0])
    assert ei.value.code == fmmlib.FMM_ERR_ARG
    with pytest.raises(fmmlib.FMMError) as ei:
        fmmlib.fmm_tree_create_batched([], [])
    assert ei.value.code == fmmlib.FMM_ERR_ARG
    t = fmmlib.fmm_tree_create_batched([100, 200], [1, 1])
    try:
        with pytest.raises(fmmlib.FMMError):
            fmmlib.fmm_tree_instance(t, 2)
        lists = fmmlib.fmm_lists_create(t)
        try:
            with pytest.raises(fmmlib.FMMError) as ei:
                fmmlib.fmm_lists_export(lists, None, None, None, None)
            assert ei.value.code in (fmmlib.FMM_ERR_ARG, fmmlib.FMM_ERR_STATE)
        finally:
            fmmlib.fmm_lists_destroy(lists)
    finally:
        fmmlib.fmm_tree_destroy(t)


# ---- the full-size batched workload ---------------------------------------------------------

@pytest.fixture(scope="module")
def big_batch(fmmlib, cuda):
    inst = W.batched_instances()
    clouds = [c for c, _ in inst]
    levels = [L for _, L in inst]
    x, y, q = _concat(clouds)
    b = fmmlib.FMMBatch(_t(x, cuda), _t(y, cuda), [c.x.shape[0] for c in clouds], levels, 0.5)
    yield clouds, levels, (x, y, q), b
    b.close()


def test_batched_workload_sampled_instances_vs_oracle(big_batch, orc, cuda):
    clouds, levels, (x, y, q), b = big_batch
    phi = b.evaluate(_t(q, cuda), 16, "mixed").cpu().numpy()
    sizes = np.array([c.x.shape[0] for c in clouds])
    pick = sorted({int(np.argmin(sizes)), int(np.argmax(sizes)), 0, 1, 2, 255, 511})
    sl = _slices(b)
    for i in pick:
        c, L = clouds[i], levels[i]
        perm, rects, lb, woff, widx, soff, sidx = b.export_instance(i)
        operm, orects, olb = orc.tree(c.x, c.y, L)
        assert np.array_equal(perm.cpu().numpy(), operm)
        assert np.array_equal(rects.cpu().numpy(), orects)
        owoff, owidx, osoff, osidx = orc.lists(orects, L, 0.5)
        assert np.array_equal(widx.cpu().numpy().astype(np.int64), owidx)
        assert np.array_equal(sidx.cpu().numpy().astype(np.int64), osidx)
        a, e = sl[i]
        ref = orc.fmm(c.x, c.y, c.q, L, 16, 0.5)
        assert relerr(phi[a:e], ref) <= TOL_MIXED, (i, c.name, c.x.shape[0], L)


def test_batched_workload_every_instance_vs_direct(big_batch, orc, cuda):
    # every instance on 24 sampled targets against the direct sum: catches any mixing between
    # instances; the bound is the truncation error at p = 16, theta = 1/2 plus rounding
    clouds, levels, (x, y, q), b = big_batch
    phi = b.evaluate(_t(q, cuda), 16, "mixed").cpu().numpy()
    worst = 0.0
    for i, ((a, e), c) in enumerate(zip(_slices(b), clouds)):
        tg = W.sample_targets(c.x.shape[0], 24, 7000 + i)
        ref = orc.direct(c.x, c.y, c.q, tg, nthreads=0)
        err = float(np.max(np.abs(phi[a:e][tg] - ref)) / np.max(np.abs(ref)))
        worst = max(worst, err)
    assert worst <= 2e-5
