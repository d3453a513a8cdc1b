"""Pins of the oracle's optional parent-level interactions (Section 4's structural optimisation),
on the CPU: every merged entry stands for exactly four weak siblings whose parent satisfies the
criterion, the interactions are still partitioned exactly once (checked point pair by point
pair), fewer shifts are needed, and the potentials keep the accuracy of the plain method."""
import numpy as np
import pytest

import oracle
from paper_1006_2269_gb300 import workloads as W

F = oracle.PARENT_FLAG


def _level_of(g):
    l = 0
    while (4 ** (l + 1) - 1) // 3 <= g:
        l += 1
    return l


@pytest.mark.parametrize("maker,L", [(lambda: W.uniform(4 ** 4 * 6, 41), 4), (lambda: W.clusters(6000, 42), 4),
                                     (lambda: W.normal(3000, 43), 3)])
def test_merge_rule(maker, L):
    c = maker()
    _, rects, _ = oracle.tree(c.x, c.y, L)
    cen, rad = oracle.geometry(rects)
    pw, pidx, ps, psi = oracle.lists(rects, L, 0.5)
    mw, midx, ms, msi = oracle.lists(rects, L, 0.5, parents=True)
    assert np.array_equal(ps, ms) and np.array_equal(psi, msi)  # strong lists untouched
    merged = 0
    for g in range(len(pw) - 1):
        plain = list(pidx[pw[g]:pw[g + 1]])
        new = list(midx[mw[g]:mw[g + 1]])
        # expanding every merged entry into its four children gives back the plain list
        exp = []
        for v in new:
            if v & F:
                k = v & ~F
                exp += [4 * k, 4 * k + 1, 4 * k + 2, 4 * k + 3]
                merged += 1
                l = _level_of(g)
                P = (4 ** (l - 1) - 1) // 3 + k
                assert oracle.theta_weak(cen[P], rad[P], cen[g], rad[g], 0.5)
            else:
                exp.append(v)
        assert exp == plain
    assert merged > 0


def test_merged_potentials_keep_accuracy():
    c = W.clusters(8000, 44)
    ref = oracle.direct(c.x, c.y, c.q)
    for p in (10, 20):
        plain = oracle.fmm(c.x, c.y, c.q, 4, p, 0.5)
        merged = oracle.fmm(c.x, c.y, c.q, 4, p, 0.5, parents=True)
        e_plain = np.max(np.abs(plain - ref)) / np.max(np.abs(ref))
        e_merged = np.max(np.abs(merged - ref)) / np.max(np.abs(ref))
        assert e_merged <= 4 * max(e_plain, 1e-14)
        assert e_merged <= 4 * 0.5 ** (p + 1) / 0.25


def test_merged_every_pair_once_small():
    # every ordered pair of points is handled exactly once: by one weak interaction (a plain or a
    # parent entry) or by the near field of the finest level
    c = W.uniform(4 ** 3 * 5, 45)
    L = 3
    perm, rects, lb = oracle.tree(c.x, c.y, L)
    mw, midx, ms, msi = oracle.lists(rects, L, 0.5, parents=True)
    n = c.x.shape[0]
    # box of every point at every level
    leaf = np.empty(n, np.int64)
    for b in range(4 ** L):
        leaf[perm[lb[b]:lb[b + 1]]] = b
    anc = [leaf // 4 ** (L - l) for l in range(L + 1)]
    count = np.zeros((n, n), np.int32)
    for l in range(1, L + 1):
        base = (4 ** l - 1) // 3
        for b in range(4 ** l):
            g = base + b
            tgt = np.where(anc[l] == b)[0]
            for v in midx[mw[g]:mw[g + 1]]:
                if v & F:
                    src = np.where(anc[l - 1] == (v & ~F))[0]
                else:
                    src = np.where(anc[l] == v)[0]
                count[np.ix_(tgt, src)] += 1
    base = (4 ** L - 1) // 3
    for b in range(4 ** L):
        tgt = np.where(anc[L] == b)[0]
        for v in msi[ms[base + b]:ms[base + b + 1]]:
            src = np.where(anc[L] == v)[0]
            count[np.ix_(tgt, src)] += 1
    np.fill_diagonal(count, 1)
    assert np.all(count == 1)
