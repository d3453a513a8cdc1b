"""Failure detection without a sanitizer: fmm_validate on every kind of built structure, the
export / import round trip of lists (resuming without a rebuild), and host-injected corruptions
of imported lists, each reported by the check it breaks -- no kernel ever evaluates them."""
import numpy as np
import pytest

from paper_1006_2269_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def _t(a, dev):
    import torch
    return torch.as_tensor(np.ascontiguousarray(a), device=dev)


@pytest.mark.parametrize("kind", ["clusters", "parents", "exchange", "uniform_mesh", "unit_root", "tiny"])
def test_validate_accepts_built_structures(fmmlib, cuda, kind):
    c = W.clusters(30000, 91) if kind != "tiny" else W.uniform(40, 92)
    L = 5 if kind != "tiny" else 0
    opt = {"parents": dict(parents=True), "exchange": dict(exchange=True, parents=True),
           "uniform_mesh": dict(mesh="uniform"), "unit_root": dict(mesh="uniform", root=(-6.0, -6.0, 12.0))}.get(kind, {})
    f = fmmlib.FMM(_t(c.x, cuda), _t(c.y, cuda), L, 0.5, **opt)
    try:
        fmmlib.fmm_validate(f.tree, f.lists)
        fmmlib.fmm_validate(f.tree)
    finally:
        f.close()


def test_validate_a_forest(fmmlib, cuda):
    clouds = [W.clusters(20000, 93), W.uniform(3000, 94), W.uniform(40, 95)]
    x = np.concatenate([c.x for c in clouds])
    y = np.concatenate([c.y for c in clouds])
    b = fmmlib.FMMBatch(_t(x, cuda), _t(y, cuda), [c.x.shape[0] for c in clouds], [5, 3, 0], 0.5, parents=True)
    try:
        fmmlib.fmm_validate(b.tree, b.lists)
    finally:
        b.close()


@pytest.fixture()
def built(fmmlib, cuda):
    c = W.clusters(30000, 96)
    f = fmmlib.FMM(_t(c.x, cuda), _t(c.y, cuda), 5, 0.5, parents=True)
    woff, widx, soff, sidx = (a.clone() for a in f.export_lists())
    yield c, f, woff, widx, soff, sidx
    f.close()


def _fresh_lists(fmmlib, f, parents=True):
    w, s = f.counts
    l = fmmlib.fmm_lists_create(f.tree, w + 16, s + 16)
    if parents:
        fmmlib.fmm_lists_set_mode(l, fmmlib.FMM_LISTS_PARENTS)
    return l


def test_import_round_trip(fmmlib, cuda, built):
    import torch
    c, f, woff, widx, soff, sidx = built
    q = _t(c.q, cuda)
    ref = f.evaluate(q, 17, "fp64").cpu().numpy()
    l = _fresh_lists(fmmlib, f)
    try:
        fmmlib.fmm_lists_import(l, 0, woff, widx, soff, sidx)
        fmmlib.fmm_validate(f.tree, l)
        phi = torch.empty(c.x.size, dtype=torch.float64, device=cuda)
        fmmlib.fmm_evaluate(f.tree, l, q, 17, fmmlib.FMM_MODE_FP64, phi)
        fmmlib.fmm_sync_status(f.tree, l)
        got = phi.cpu().numpy()
        assert np.max(np.abs(got - ref)) <= 1e-13 * np.max(np.abs(ref))
    finally:
        fmmlib.fmm_lists_destroy(l)


@pytest.mark.parametrize("what,message", [
    ("weak_index_out_of_level", "weak-list entries"),
    ("parent_index_out_of_level", "weak-list entries"),
    ("strong_index_negative", "strong-list entries"),
    ("offsets_not_monotone", "list offsets"),
    ("count_beyond_capacity", None),
])
def test_import_corruption_is_reported(fmmlib, cuda, built, what, message):
    c, f, woff, widx, soff, sidx = built
    w, wi, s, si = woff.clone(), widx.clone(), soff.clone(), sidx.clone()
    L = 5
    base = (4 ** L - 1) // 3
    if what == "weak_index_out_of_level":
        e = int(w[base].item())  # an entry of a leaf
        wi[e] = 4 ** L
    elif what == "parent_index_out_of_level":
        e = int(w[base].item())
        wi[e] = (4 ** (L - 1)) | fmmlib.FMM_PARENT_FLAG
    elif what == "strong_index_negative":
        si[int(s[base].item())] = -3
    elif what == "offsets_not_monotone":
        w[base + 7] = w[base + 6] - 1
    elif what == "count_beyond_capacity":
        w[-1] = int(w[-1].item()) + 10 ** 7
    l = _fresh_lists(fmmlib, f)
    try:
        if message is None:
            with pytest.raises(fmmlib.FMMError) as ei:
                fmmlib.fmm_lists_import(l, 0, w, wi, s, si)
            assert ei.value.code == fmmlib.FMM_ERR_CAPACITY
            return
        fmmlib.fmm_lists_import(l, 0, w, wi, s, si)
        with pytest.raises(fmmlib.FMMError) as ei:
            fmmlib.fmm_validate(f.tree, l)
        assert ei.value.code == fmmlib.FMM_ERR_STATE and message in str(ei.value)
    finally:
        fmmlib.fmm_lists_destroy(l)


def test_bounded_wait_gives_up_and_the_context_survives(fmmlib, orc, cuda):
    # the tensor-core M2L's bounded wait, on an mbarrier that nothing completes
    with pytest.raises(fmmlib.FMMError) as ei:
        fmmlib.fmm_selftest_bounded_wait(4096)
    assert ei.value.code == fmmlib.FMM_ERR_TIMEOUT
    # and the device goes on evaluating normally
    c = W.uniform(5000, 97)
    f = fmmlib.FMM(_t(c.x, cuda), _t(c.y, cuda), 3, 0.5)
    try:
        got = f.evaluate(_t(c.q, cuda), 16, "fp64").cpu().numpy()
        ref = orc.fmm(c.x, c.y, c.q, 3, 16, 0.5)
        assert np.max(np.abs(got - ref)) <= 1e-12 * np.max(np.abs(ref))
    finally:
        f.close()


def test_queue_wait_gives_up_and_the_context_survives(fmmlib, orc, cuda):
    # the persistent upward pass with a dependency that never completes: every waiting item
    # gives up after its tries, the launch ends, and the tree then evaluates normally
    c = W.clusters(20000, 98)
    f = fmmlib.FMM(_t(c.x, cuda), _t(c.y, cuda), 4, 0.5)
    try:
        with pytest.raises(fmmlib.FMMError) as ei:
            fmmlib.fmm_selftest_queue_timeout(f.tree, 4096)
        assert ei.value.code == fmmlib.FMM_ERR_TIMEOUT
        got = f.evaluate(_t(c.q, cuda), 16, "fp64").cpu().numpy()
        ref = orc.fmm(c.x, c.y, c.q, 4, 16, 0.5)
        assert np.max(np.abs(got - ref)) <= 1e-12 * np.max(np.abs(ref))
    finally:
        f.close()
