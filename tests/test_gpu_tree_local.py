"""The median tree's lowest levels split inside one block per box (boxes of at most
TREE_LOCAL_CAP = 4096 points) against the oracle, bit for bit: at the capacity boundary (boxes of
exactly 4096 and of 4097 points), with every level inside blocks, with none (leaves larger than a
block), with coincident points, and in a forest mixing all of these, built alone and inside the
two-stream step (whose list build waits for each level's geometry)."""
import numpy as np
import pytest

from paper_1006_2269_gb300 import workloads as W

pytestmark = pytest.mark.gpu

CAP = 4096


def _t(a, dev):
    import torch
    return torch.as_tensor(np.ascontiguousarray(a), device=dev)


def _dupes(n, seed):
    c = W.uniform(n, seed)
    return W.Cloud(np.round(c.x * 8) / 8, np.round(c.y * 8) / 8, c.q, "dupes")


def _first_local_level(n, L):
    lg = 0
    while lg < L and -(-n // 4 ** lg) > CAP:
        lg += 1
    return lg


CASES = [
    ("box_4096", lambda: W.uniform(4 * CAP, 21), 4),             # level-1 boxes of exactly 4096
    ("box_4097", lambda: W.clusters(4 * CAP + 1, 22), 4),        # 4097: one level further down
    ("all_local", lambda: W.normal(CAP, 23), 5),                 # the whole tree in one block
    ("none_local", lambda: W.uniform(5 * CAP, 24), 1),           # leaves of 5120 points
    ("dupes_local", lambda: _dupes(3000, 25), 3),
    ("deep", lambda: W.rings_plummer(70000, 26), 7),
]


def _check_tree(perm, rects, lb, c, L, orc):
    operm, orects, olb = orc.tree(c.x, c.y, L)
    assert np.array_equal(perm, operm)
    assert np.array_equal(lb.astype(np.int64), olb)
    assert np.array_equal(rects, orects)
    return orects


@pytest.mark.parametrize("k", range(len(CASES)))
def test_tree_and_lists_bit_exact(fmmlib, orc, cuda, k):
    name, make, L = CASES[k]
    c = make()
    lg = _first_local_level(c.x.size, L)
    assert {"box_4096": 1, "box_4097": 2, "all_local": 0, "none_local": 1}.get(name, lg) == lg
    f = fmmlib.FMM(_t(c.x, cuda), _t(c.y, cuda), L, 0.5)
    try:
        perm, rects, lb = (a.cpu().numpy() for a in f.export_tree())
        orects = _check_tree(perm, rects, lb, c, L, orc)
        woff, widx, soff, sidx = (a.cpu().numpy().astype(np.int64) for a in f.export_lists())
        ow, oi, os_, osi = orc.lists(orects, L, 0.5)
        assert np.array_equal(woff, ow) and np.array_equal(widx, oi)
        assert np.array_equal(soff, os_) and np.array_equal(sidx, osi)
        fmmlib.fmm_sync_status(f.tree, f.lists)
    finally:
        f.close()


def test_forest_of_mixed_split_levels_and_step(fmmlib, orc, cuda):
    import torch
    picks = [CASES[0], CASES[1], CASES[2], CASES[3], CASES[4]]
    clouds = [make() for _, make, _ in picks] + [W.uniform(40, 27)]
    levels = [L for _, _, L in picks] + [0]
    x = np.concatenate([c.x for c in clouds])
    y = np.concatenate([c.y for c in clouds])
    q = np.concatenate([c.q for c in clouds])
    xd, yd, qd = _t(x, cuda), _t(y, cuda), _t(q, cuda)
    b = fmmlib.FMMBatch(xd, yd, [c.x.size for c in clouds], levels, 0.5)
    try:
        for i, (c, L) in enumerate(zip(clouds, levels)):
            perm, rects, lb = (a.cpu().numpy() for a in b.export_instance(i)[:3])
            _check_tree(perm, rects, lb, c, L, orc)
        phi = torch.empty(x.size, dtype=torch.float64, device=cuda)
        for _ in range(2):  # the step rebuilds the tree; the lists follow each level's geometry
            fmmlib.fmm_step(b.tree, b.lists, xd, yd, 0.5, qd, 17, fmmlib.FMM_MODE_FP64, phi)
        fmmlib.fmm_sync_status(b.tree, b.lists)
        got = phi.cpu().numpy()
        for d, c, L in zip(b.inst, clouds, levels):
            ref = orc.fmm(c.x, c.y, c.q, L, 17, 0.5)
            err = np.max(np.abs(got[d["p0"]:d["p0"] + d["n"]] - ref)) / np.max(np.abs(ref))
            assert err <= 1e-12
        for i, (c, L) in enumerate(zip(clouds, levels)):
            perm, rects, lb = (a.cpu().numpy() for a in b.export_instance(i)[:3])
            _check_tree(perm, rects, lb, c, L, orc)
    finally:
        b.close()
