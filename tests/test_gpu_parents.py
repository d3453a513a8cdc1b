"""Parent-level interactions (Section 4's optional structural optimisation) on the GPU against
the oracle in the same mode: merged weak lists bit for bit, potentials within 1e-12 (binary64)
and 1e-6 (mixed, both M2L kernels), a forest, and fewer shifts than the plain lists."""
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
    ("uniform", lambda: W.uniform(4 ** 5 * 6, 51), 5),
    ("clusters", lambda: W.clusters(30011, 52), 5),
    ("normal", lambda: W.normal(12345, 53), 4),
    ("circle", lambda: W.circle(20000, 54), 5),
    ("ragged_L2", lambda: W.uniform(4 ** 2 + 5, 55), 2),
]


@pytest.fixture(scope="module")
def built(fmmlib, cuda):
    out = {}
    for name, make, L in CASES:
        c = make()
        out[name] = (c, L, fmmlib.FMM(_t(c.x, cuda), _t(c.y, cuda), L, 0.5, parents=True))
    yield out
    for _, _, f in out.values():
        f.close()


@pytest.mark.parametrize("theta", [0.5, 0.3])
@pytest.mark.parametrize("name", [c[0] for c in CASES])
def test_merged_lists_bit_exact(built, orc, cuda, name, theta):
    c, L, f = built[name]
    if theta != 0.5:
        f.rebuild(_t(c.x, cuda), _t(c.y, cuda), theta=theta)
    try:
        woff, widx, soff, sidx = (a.cpu().numpy().astype(np.int64) for a in f.export_lists())
        _, rects, _ = orc.tree(c.x, c.y, L)
        ow, oi, os_, osi = orc.lists(rects, L, theta, parents=True)
        assert np.array_equal(woff, ow) and np.array_equal(widx, oi)
        assert np.array_equal(soff, os_) and np.array_equal(sidx, osi)
        pw, _, _, _ = orc.lists(rects, L, theta)
        if L >= 3:
            assert ow[-1] < pw[-1]  # fewer shifts
    finally:
        if theta != 0.5:
            f.rebuild(_t(c.x, cuda), _t(c.y, cuda), theta=0.5)


@pytest.mark.parametrize("name", [c[0] for c in CASES])
@pytest.mark.parametrize("mode,p,tol,kind", [("fp64", 17, 1e-12, 0), ("mixed", 20, 1e-6, 1), ("mixed", 20, 1e-6, 2),
                                             ("mixed", 30, 1e-6, 0)])
def test_merged_potentials(built, orc, fmmlib, cuda, name, mode, p, tol, kind):
    c, L, f = built[name]
    fmmlib.fmm_set_m2l_kernel(f.tree, kind)
    try:
        got = f.evaluate(_t(c.q, cuda), p, mode).cpu().numpy()
    finally:
        fmmlib.fmm_set_m2l_kernel(f.tree, 0)
    ref = orc.fmm(c.x, c.y, c.q, L, p, 0.5, parents=True)
    assert relerr(got, ref) <= tol


def test_merged_forest(fmmlib, orc, cuda):
    clouds = [W.uniform(5000, 61), W.clusters(20000, 62), W.uniform(40, 63)]
    levels = [4, 5, 0]
    x = np.concatenate([c.x for c in clouds])
    y = np.concatenate([c.y for c in clouds])
    q = np.concatenate([c.q for c in clouds])
    b = fmmlib.FMMBatch(_t(x, cuda), _t(y, cuda), [c.x.shape[0] for c in clouds], levels, 0.5, parents=True)
    try:
        for i, (c, L) in enumerate(zip(clouds, levels)):
            _, rects, _, woff, widx, soff, sidx = b.export_instance(i)
            ow, oi, _, _ = orc.lists(rects.cpu().numpy(), L, 0.5, parents=True)
            assert np.array_equal(woff.cpu().numpy().astype(np.int64), ow)
            assert np.array_equal(widx.cpu().numpy().astype(np.int64), oi)
        phi = b.evaluate(_t(q, cuda), 16, "fp64").cpu().numpy()
        for d, c, L in zip(b.inst, clouds, levels):
            ref = orc.fmm(c.x, c.y, c.q, L, 16, 0.5, parents=True)
            assert relerr(phi[d["p0"]:d["p0"] + d["n"]], ref) <= 1e-12
    finally:
        b.close()


def test_mode_switch_on_the_same_lists(fmmlib, orc, cuda):
    # parents -> plain -> parents on one lists object: each build matches the oracle in its mode
    c = W.clusters(20000, 64)
    L = 5
    f = fmmlib.FMM(_t(c.x, cuda), _t(c.y, cuda), L, 0.7)  # capacities sized by the plain lists
    try:
        _, rects, _ = orc.tree(c.x, c.y, L)
        for par in (True, False, True):
            fmmlib.fmm_lists_set_mode(f.lists, fmmlib.FMM_LISTS_PARENTS if par else fmmlib.FMM_LISTS_PLAIN)
            fmmlib.fmm_interaction_lists(f.tree, f.lists, 0.7)
            woff, widx, soff, sidx = (a.cpu().numpy().astype(np.int64) for a in f.export_lists())
            ow, oi, os_, osi = orc.lists(rects, L, 0.7, parents=par)
            assert np.array_equal(woff, ow) and np.array_equal(widx, oi)
            assert np.array_equal(soff, os_) and np.array_equal(sidx, osi)
    finally:
        f.close()
