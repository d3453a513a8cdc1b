"""The binary32 near field's two work shapes (two or four targets of a leaf per lane) against
the oracle and against each other, on leaves from a handful of points to the 64-point limit of
the leaf-pair kernel, with ragged leaf sizes and the leaf-with-itself pairs."""
import numpy as np
import pytest

from paper_1006_2269_gb300 import workloads as W

pytestmark = pytest.mark.gpu

TOL_MIXED = 1e-6


def _t(a, dev):
    import torch
    return torch.as_tensor(np.ascontiguousarray(a), device=dev)


def relerr(a, ref):
    return float(np.max(np.abs(a - ref)) / np.max(np.abs(ref)))


CASES = [
    ("uniform_leaf3", lambda: W.uniform(4 ** 4 * 3 + 1, 501), 4),      # leaves of 3 and 4 points
    ("clusters_leaf16", lambda: W.clusters(4 ** 5 * 16 + 77, 502), 5),  # 16 and 17
    ("circle_leaf40", lambda: W.circle(4 ** 4 * 40 + 9, 503), 4),       # 40 and 41
    ("normal_leaf64", lambda: W.normal(4 ** 4 * 64, 504), 4),           # exactly 64
]


@pytest.mark.parametrize("name", [c[0] for c in CASES])
def test_near_field_targets_per_lane(fmmlib, orc, cuda, name):
    make, L = {c[0]: (c[1], c[2]) for c in CASES}[name]
    c = make()
    p = 16
    f = fmmlib.FMM(_t(c.x, cuda), _t(c.y, cuda), L, 0.5)
    try:
        q = _t(c.q, cuda)
        out = {}
        for nt in (2, 4):
            fmmlib.fmm_set_near_shape(f.tree, nt)
            assert fmmlib.fmm_get_near_shape(f.tree) == nt
            out[nt] = f.evaluate(q, p, "mixed").cpu().numpy()
        fmmlib.fmm_set_near_shape(f.tree, 0)
        assert fmmlib.fmm_get_near_shape(f.tree) == 0
    finally:
        f.close()
    ref = orc.fmm(c.x, c.y, c.q, L, p, 0.5)
    for nt in (2, 4):
        assert relerr(out[nt], ref) <= TOL_MIXED, nt
    assert relerr(out[2], out[4]) <= TOL_MIXED
