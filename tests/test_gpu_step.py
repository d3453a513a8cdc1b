"""The two-stream whole step (fmm_step: mesh, lists and evaluation with the independent parts on a
second stream) against the oracle and against the three separate calls, with the list variants
of Section 4, on a forest, replayed from a CUDA graph, and with the stage profile."""
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
    ("clusters", lambda: W.clusters(40000, 61), 5, dict()),
    ("clusters_parents", lambda: W.clusters(40000, 61), 5, dict(parents=True)),
    ("rings_exchange", lambda: W.rings_plummer(30000, 62), 5, dict(exchange=True)),
    ("big_leaves", lambda: W.normal(4 ** 3 * 90, 63), 3, dict()),  # 90 points per leaf: general kernel
    ("L0", lambda: W.uniform(60, 64), 0, dict()),
]


@pytest.mark.parametrize("k", range(len(CASES)))
@pytest.mark.parametrize("mode,p,tol", [("fp64", 17, 1e-12), ("mixed", 20, 1e-6)])
def test_step_matches_oracle_and_separate_calls(fmmlib, orc, cuda, k, mode, p, tol):
    import torch
    name, make, L, opt = CASES[k]
    c = make()
    x, y, q = _t(c.x, cuda), _t(c.y, cuda), _t(c.q, cuda)
    f = fmmlib.FMM(x, y, L, 0.5, **opt)
    try:
        m = fmmlib.FMM_MODE_FP64 if mode == "fp64" else fmmlib.FMM_MODE_MIXED
        sep = f.evaluate(q, p, mode).cpu().numpy()
        phi = torch.empty(c.x.size, dtype=torch.float64, device=cuda)
        for _ in range(2):
            fmmlib.fmm_step(f.tree, f.lists, x, y, 0.5, q, p, m, phi)
        fmmlib.fmm_sync_status(f.tree, f.lists)
        got = phi.cpu().numpy()
        ref = orc.fmm(c.x, c.y, c.q, L, p, 0.5, parents=opt.get("parents", False), swap=opt.get("exchange", False))
        assert relerr(got, ref) <= tol
        # binary32 atomics add in a different order on every run: the two agree to the mixed tolerance
        assert relerr(got, sep) <= (1e-12 if mode == "fp64" else 1e-6)
    finally:
        f.close()


def test_step_on_a_forest(fmmlib, orc, cuda):
    import torch
    clouds = [W.clusters(20000, 65), W.uniform(3000, 66), W.circle(9000, 67)]
    levels = [5, 3, 4]
    x = np.concatenate([c.x for c in clouds])
    y = np.concatenate([c.y for c in clouds])
    q = np.concatenate([c.q for c in clouds])
    b = fmmlib.FMMBatch(_t(x, cuda), _t(y, cuda), [c.x.shape[0] for c in clouds], levels, 0.5)
    try:
        phi = torch.empty(x.size, dtype=torch.float64, device=cuda)
        fmmlib.fmm_step(b.tree, b.lists, _t(x, cuda), _t(y, cuda), 0.5, _t(q, cuda), 20, fmmlib.FMM_MODE_MIXED, phi)
        got = phi.cpu().numpy()
        for d, c, L in zip(b.inst, clouds, levels):
            assert relerr(got[d["p0"]:d["p0"] + d["n"]], orc.fmm(c.x, c.y, c.q, L, 20, 0.5)) <= 1e-6
    finally:
        b.close()


def test_step_graph_replay(fmmlib, orc, cuda):
    import torch
    c = W.clusters(50000, 68)
    L = 6
    x, y, q = _t(c.x, cuda), _t(c.y, cuda), _t(c.q, cuda)
    f = fmmlib.FMM(x, y, L, 0.5, parents=True)
    try:
        phi = torch.empty(c.x.size, dtype=torch.float64, device=cuda)
        side = torch.cuda.Stream()
        side.wait_stream(torch.cuda.current_stream())
        with torch.cuda.stream(side):  # first call outside capture: creates the second stream
            fmmlib.fmm_step(f.tree, f.lists, x, y, 0.5, q, 20, fmmlib.FMM_MODE_MIXED, phi)
        torch.cuda.current_stream().wait_stream(side)
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g):
            fmmlib.fmm_step(f.tree, f.lists, x, y, 0.5, q, 20, fmmlib.FMM_MODE_MIXED, phi)
        phi.zero_()
        g.replay()
        torch.cuda.synchronize()
        fmmlib.fmm_sync_status(f.tree, f.lists)
        ref = orc.fmm(c.x, c.y, c.q, L, 20, 0.5, parents=True)
        assert relerr(phi.cpu().numpy(), ref) <= 1e-6
        # new strengths through the same graph
        q2 = _t(np.random.default_rng(69).uniform(-1, 1, c.x.size), cuda)
        q.copy_(q2)
        g.replay()
        torch.cuda.synchronize()
        assert relerr(phi.cpu().numpy(), orc.fmm(c.x, c.y, q2.cpu().numpy(), L, 20, 0.5, parents=True)) <= 1e-6
    finally:
        f.close()


@pytest.mark.parametrize("exchange,mode", [(False, "mixed"), (True, "mixed"), (True, "split"), (True, "fp64")])
def test_step_profile_has_every_stage(fmmlib, cuda, exchange, mode):
    # every stage is timed once per step; the role-exchange stage only with exchange lists
    import torch
    c = W.clusters(30000, 70)
    x, y, q = _t(c.x, cuda), _t(c.y, cuda), _t(c.q, cuda)
    f = fmmlib.FMM(x, y, 5, 0.5, exchange=exchange)
    m = {"mixed": fmmlib.FMM_MODE_MIXED, "split": fmmlib.FMM_MODE_SPLIT, "fp64": fmmlib.FMM_MODE_FP64}[mode]
    try:
        phi = torch.empty(c.x.size, dtype=torch.float64, device=cuda)
        fmmlib.fmm_step(f.tree, f.lists, x, y, 0.5, q, 20, m, phi)
        torch.cuda.synchronize()
        fmmlib.fmm_profile_read()
        fmmlib.fmm_profile_enable(True)
        for _ in range(3):
            fmmlib.fmm_step(f.tree, f.lists, x, y, 0.5, q, 20, m, phi)
        torch.cuda.synchronize()
        fmmlib.fmm_profile_enable(False)
        prof = fmmlib.fmm_profile_read()
        for st in fmmlib.STAGES:
            if st == "exchange" and not exchange:  # plain lists: no P2L or M2P
                assert prof[st][1] == 0, st
                continue
            assert prof[st][1] == 3 and prof[st][0] > 0, st
    finally:
        f.close()
