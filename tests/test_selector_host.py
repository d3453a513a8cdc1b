"""Host-side logic of the parameter selector (no GPU): the plain rule, classes, labels."""
import math

import pytest

from paper_1006_2269_gb300 import selector as S


def test_fallback_rule():
    # smallest p with 2^-(p+1) * 4 <= tol, about 20 points per leaf
    assert S.fallback_params(10 ** 6, 1e-6) == (8, 21)
    assert S.fallback_params(20000, 1e-3) == (5, 11)
    assert S.fallback_params(300, 1e-9) == (4, 31)
    for tol in (1e-3, 1e-6, 1e-9):
        _, p = S.fallback_params(10 ** 5, tol)
        assert 0.5 ** (p + 1) * 4 <= tol < 0.5 ** p * 4


def test_classes_round_trip():
    seen = set()
    for L in range(S.LMIN, S.LMAX + 1):
        for p in range(S.PMIN, S.PMAX + 1):
            c = S.class_of(L, p)
            assert 0 <= c < S.NCLASS and S.params_of(c) == (L, p)
            seen.add(c)
    assert len(seen) == S.NCLASS == 225


def test_label_picks_fastest_feasible():
    tab = [(5, 10, 1.0, 3e-4), (5, 12, 1.2, 2e-5), (6, 10, 0.8, 5e-3), (6, 14, 0.9, 1e-7)]
    assert S.label(tab, 1e-3) == S.class_of(6, 14)
    assert S.label(tab, 1e-2) == S.class_of(6, 10)
    assert S.label(tab, 1e-9) == S.class_of(6, 14)  # nothing meets it: the most accurate


@pytest.mark.parametrize("n", [10 ** 4, 37000, 2 * 10 ** 5, 10 ** 6])
def test_candidates_are_feasible(n):
    Ls = S.candidate_levels(n)
    assert Ls and all(S.LMIN <= L <= S.LMAX and 4 ** L <= n for L in Ls)
    assert S.probe_levels(n) <= S.max_levels(n)
    for tol in S.TOLS:
        assert all(S.PMIN <= p <= S.PMAX for p in S.candidate_ps(tol))


def test_probe_depth():
    # about 16 points per leaf inside the training range (N <= 1e6), never deeper than its deepest
    for n in (10 ** 4, 37000, 2 * 10 ** 5, 10 ** 6):
        assert S.probe_levels(n) == math.floor(math.log(n / 16) / math.log(4))
    assert S.probe_levels(10 ** 6) == S.PROBE_LMAX
    assert S.probe_levels(1 << 20) == S.probe_levels(1 << 24) == S.PROBE_LMAX


def test_committed_weights_on_benchmark_cloud():
    # the committed network on the 2^20-point clustered cloud (features of the oracle's probe
    # tree): the trees it picks hold 16 to 64 points per leaf, as the labels of the training
    # sets near 1e6 points do
    import numpy as np
    import oracle as orc
    from oracle import mlp as M
    from paper_1006_2269_gb300 import workloads as W
    params = np.fromfile(S.WEIGHTS + ".f32", dtype=np.float32).astype(np.float64)
    c = W.mixed_1m_cloud()
    n = c.x.shape[0]
    L = S.probe_levels(n)
    _, rects, _ = orc.tree(c.x, c.y, L)
    for tol in S.TOLS:
        prob = M.forward(params, M.features(rects, L, n, tol)[None])[0]
        levels, p = S.params_of(int(np.argmax(prob)))
        assert levels in (7, 8), (tol, levels, p)


def test_centre_level_is_half_up_rounding():
    # the integer rule equals round(log4(N / 32)) with halves rounded up, away from exact ties
    # checked against the logarithm; at the ties (N = 2^(2k+6)) it gives the upper level
    for n in [300, 1000, 12345, 10 ** 4, 37000, 2 * 10 ** 5, 10 ** 6, 3 * 10 ** 6, 2 ** 24 + 3]:
        v = math.log(n / 32.0) / math.log(4.0)
        assert S.centre_level(n) == math.floor(v + 0.5), n
    for k in range(2, 10):
        assert S.centre_level(2 ** (2 * k + 6)) == k + 1
    assert S.candidate_levels(1 << 20) == [6, 7, 8, 9]
