"""The tensor-core M2L (tcgen05, split-tf32 products) against the oracle and against the SIMT
binary32 M2L on the same trees and lists.

Both kernels compute the same shifts in different arithmetic, so the potentials agree to the
binary32 rounding level; both must stay within the mixed path's tolerance of the oracle.  Cases
cover every p bucket of the tensor-core kernel (K = 24 for p <= 23, K = 32 for p <= 31), the
fallback to the SIMT kernel above, partial last tiles, level counts 1..8 and forests.
"""
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
    ("uniform_L1", lambda: W.uniform(300, 401), 1),
    ("clusters", lambda: W.clusters(30011, 402), 5),
    ("circle", lambda: W.circle(20000, 403), 5),
    ("rings", lambda: W.rings_plummer(40000, 404), 6),
    ("normal_ragged", lambda: W.normal(4 ** 4 * 7 + 3, 405), 4),
]


@pytest.mark.parametrize("p", [5, 16, 20, 23, 24, 31, 34])
@pytest.mark.parametrize("name", [c[0] for c in CASES])
def test_tensor_core_m2l(fmmlib, orc, cuda, name, p):
    make, L = {c[0]: (c[1], c[2]) for c in CASES}[name]
    c = make()
    f = fmmlib.FMM(_t(c.x, cuda), _t(c.y, cuda), L, 0.5)
    try:
        q = _t(c.q, cuda)
        fmmlib.fmm_set_m2l_kernel(f.tree, fmmlib.FMM_M2L_TENSOR)
        tc = f.evaluate(q, p, "mixed").cpu().numpy()
        fmmlib.fmm_set_m2l_kernel(f.tree, fmmlib.FMM_M2L_SIMT)
        simt = f.evaluate(q, p, "mixed").cpu().numpy()
        fmmlib.fmm_set_m2l_kernel(f.tree, fmmlib.FMM_M2L_AUTO)
    finally:
        f.close()
    ref = orc.fmm(c.x, c.y, c.q, L, p, 0.5)
    assert relerr(tc, ref) <= TOL_MIXED
    assert relerr(simt, ref) <= TOL_MIXED
    assert relerr(tc, simt) <= TOL_MIXED


def test_tensor_core_m2l_forest(fmmlib, orc, cuda):
    clouds = [W.uniform(5000, 411), W.clusters(20000, 412), W.circle(3000, 413), W.uniform(40, 414)]
    levels = [4, 5, 3, 0]
    x = np.concatenate([c.x for c in clouds])
    y = np.concatenate([c.y for c in clouds])
    q = np.concatenate([c.q for c in clouds])
    b = fmmlib.FMMBatch(_t(x, cuda), _t(y, cuda), [c.x.shape[0] for c in clouds], levels, 0.5)
    try:
        fmmlib.fmm_set_m2l_kernel(b.tree, fmmlib.FMM_M2L_TENSOR)
        phi = b.evaluate(_t(q, cuda), 18, "mixed").cpu().numpy()
        for d, c, L in zip(b.inst, clouds, levels):
            ref = orc.fmm(c.x, c.y, c.q, L, 18, 0.5)
            assert relerr(phi[d["p0"]:d["p0"] + d["n"]], ref) <= TOL_MIXED
    finally:
        b.close()


@pytest.mark.parametrize("chunk,stages", [(1, 1), (3, 2), (16, 1), (16, 2), (64, 2)])
@pytest.mark.parametrize("p", [16, 20, 30])
def test_tensor_core_m2l_tile_shapes(fmmlib, orc, cuda, chunk, stages, p):
    # every row of a tile takes `chunk` consecutive weak entries: 1 (a target change at almost
    # every entry), an odd shape whose chunks end inside target runs, the default, and chunks
    # longer than most target runs; one or two TMEM accumulator stages; p = 16, 20, 30 take the
    # exact-order kernels; a ragged last chunk in every case
    c = W.clusters(30011, 402)
    L = 5
    f = fmmlib.FMM(_t(c.x, cuda), _t(c.y, cuda), L, 0.5, parents=True)
    try:
        q = _t(c.q, cuda)
        fmmlib.fmm_set_m2l_kernel(f.tree, fmmlib.FMM_M2L_TENSOR)
        fmmlib.fmm_set_m2l_shape(f.tree, chunk, stages)
        assert fmmlib.fmm_get_m2l_shape(f.tree) == (chunk, stages)
        tc = f.evaluate(q, p, "mixed").cpu().numpy()
        fmmlib.fmm_set_m2l_kernel(f.tree, fmmlib.FMM_M2L_SIMT)
        simt = f.evaluate(q, p, "mixed").cpu().numpy()
    finally:
        f.close()
    ref = orc.fmm(c.x, c.y, c.q, L, p, 0.5, parents=True)
    assert relerr(tc, ref) <= TOL_MIXED
    assert relerr(tc, simt) <= TOL_MIXED
