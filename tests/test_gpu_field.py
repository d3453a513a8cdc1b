"""The complex field F_i = sum_{j != i} -q_j / (z_i - z_j) (the kernel of the paper's first
experiment) on the GPU against the oracle's field by the same method: binary64 within 1e-12,
mixed within 1e-6 (max-norm relative to max |F|), on the parity cases, a forest and the direct
kernel; and the method's error against the direct field falling with p at the rate the
Section 3 estimate predicts."""
import numpy as np
import pytest

from paper_1006_2269_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def _t(a, dev):
    import torch
    return torch.as_tensor(np.ascontiguousarray(a), device=dev)


def relerr(a, ref):
    return float(np.max(np.abs(a - ref)) / np.max(np.abs(ref)))


def _dupes(n=4000, seed=8):
    c = W.uniform(n, seed)
    return W.Cloud(np.round(c.x * 16) / 16, np.round(c.y * 16) / 16, c.q, "dupes")


def _collinear(n=3000, seed=9):
    c = W.uniform(n, seed)
    return W.Cloud(c.x, np.full(n, 0.25), c.q, "collinear")


CASES = [
    ("tiny_L0", lambda: W.uniform(37, 1), 0),
    ("L1", lambda: W.uniform(101, 2), 1),
    ("ragged", lambda: W.uniform(4 ** 3 + 13, 3), 3),
    ("clusters", lambda: W.clusters(30011, 5), 5),
    ("circle", lambda: W.circle(20000, 6), 5),
    ("rings", lambda: W.rings_plummer(40000, 8), 6),
    ("disc_inv_r", lambda: W.disc_inv_r(20000, 12), 5),
    ("dupes", _dupes, 3),
    ("collinear", _collinear, 4),
    ("big_leaves", lambda: W.normal(4 ** 3 * 90, 13), 3),  # 90 points per leaf: binary64 path
]


@pytest.fixture(scope="module")
def built(fmmlib, cuda):
    out = {}
    for name, make, L in CASES:
        c = make()
        out[name] = (c, L, fmmlib.FMM(_t(c.x, cuda), _t(c.y, cuda), L, 0.5))
    yield out
    for _, _, f in out.values():
        f.close()


@pytest.mark.parametrize("name", [c[0] for c in CASES])
@pytest.mark.parametrize("mode,p,tol", [("fp64", 17, 1e-12), ("mixed", 16, 1e-6), ("mixed", 20, 1e-6)])
def test_field_vs_oracle(built, orc, cuda, name, mode, p, tol):
    c, L, f = built[name]
    got = f.evaluate_field(_t(c.q, cuda), p, mode).cpu().numpy()
    ref = orc.fmm_field(c.x, c.y, c.q, L, p, 0.5)
    assert relerr(got, ref) <= tol


def test_field_forest(fmmlib, orc, cuda):
    clouds = [W.uniform(5000, 21), W.clusters(20000, 22), W.circle(3000, 23), W.uniform(40, 24)]
    levels = [4, 5, 3, 0]
    x = np.concatenate([c.x for c in clouds])
    y = np.concatenate([c.y for c in clouds])
    q = np.concatenate([c.q for c in clouds])
    b = fmmlib.FMMBatch(_t(x, cuda), _t(y, cuda), [c.x.shape[0] for c in clouds], levels, 0.5)
    try:
        for mode, tol in (("fp64", 1e-12), ("mixed", 1e-6)):
            got = b.evaluate_field(_t(q, cuda), 18, mode).cpu().numpy()
            for d, c, L in zip(b.inst, clouds, levels):
                ref = orc.fmm_field(c.x, c.y, c.q, L, 18, 0.5)
                assert relerr(got[d["p0"]:d["p0"] + d["n"]], ref) <= tol
    finally:
        b.close()


def test_direct_field_kernel(fmmlib, orc, cuda):
    import torch
    c = W.clusters(20000, 25)
    tg = W.sample_targets(c.x.shape[0], 300, 26)
    fre = torch.empty(tg.shape[0], dtype=torch.float64, device=cuda)
    fim = torch.empty(tg.shape[0], dtype=torch.float64, device=cuda)
    fmmlib.fmm_direct_field(_t(c.x, cuda), _t(c.y, cuda), _t(c.q, cuda), _t(tg, cuda), fre, fim)
    ref = orc.direct_field(c.x, c.y, c.q, tg)
    assert relerr(fre.cpu().numpy() + 1j * fim.cpu().numpy(), ref) <= 1e-13


def test_field_error_falls_with_p(fmmlib, orc, cuda):
    c = W.disc_uniform(50000, 27)
    f = fmmlib.FMM(_t(c.x, cuda), _t(c.y, cuda), 6, 0.5)
    try:
        tg = W.sample_targets(c.x.shape[0], 1000, 28)
        ref = orc.direct_field(c.x, c.y, c.q, tg)
        errs = [relerr(f.evaluate_field(_t(c.q, cuda), p, "fp64").cpu().numpy()[tg], ref) for p in (6, 12, 18, 24)]
    finally:
        f.close()
    errs = np.array(errs)
    assert np.all(errs[1:] <= errs[:-1] / 16)  # six orders: at least theta^4 per step
    assert errs[-1] < 1e-8
