"""Pins of the oracle's finest-level role exchange (Section 4's second structural optimisation),
on the CPU.

Criterion: hand values, and the exchanged test as the smaller set expanded by 1/theta about its
centre staying clear of the larger one (symmetric, Criterion 2.1 for equal radii, implied by it).

Operators: the P2L expansion evaluated inside its disc against the direct sum, within the
truncation bound of the logarithm's series, |sum_{l>p} u^l / l| <= |u|^(p+1) / ((p+1)(1-|u|)),
and M2P likewise.  Lists: the exchanged pairs and the remaining strong pairs of a leaf are the
plain strong list split in order; every exchanged pair is separated at ratio theta as seen from
the actual points (not the circles); the M2P mark goes to the larger target.  Congruent leaves
never exchange (a lattice exchanges only pairs with its narrower border leaves), nor do the
touching leaves of trees with one level.  The method: against the direct sum within the
Section 3 estimate, converging in p, for the potential and the field.
"""
import numpy as np
import pytest

import oracle
from paper_1006_2269_gb300 import workloads as W


def _disc_and_annulus(seed, m_src=40, m_tgt=25, r_tgt=0.3, r_in=1.2, r_out=2.0):
    g = np.random.default_rng(seed)
    a = g.uniform(0, 2 * np.pi, m_src)
    rad = g.uniform(r_in, r_out, m_src)
    src = rad * np.exp(1j * a)
    tgt = r_tgt * np.sqrt(g.uniform(0, 1, m_tgt)) * np.exp(1j * g.uniform(0, 2 * np.pi, m_tgt))
    q = g.normal(size=m_src)
    return src, tgt, q


def test_swapped_criterion_hand_values():
    # R = 2, r = 0.5, theta = 1/4: swapped iff 0.5 + 0.5 <= 0.25 d, i.e. d >= 4 (plain: d >= 8.5)
    assert oracle.theta_swapped((0, 0), 2.0, (4.0, 0), 0.5, 0.25)
    assert oracle.theta_swapped((0, 0), 0.5, (0, -4.0), 2.0, 0.25)  # argument order does not matter
    assert not oracle.theta_swapped((0, 0), 2.0, (3.99, 0), 0.5, 0.25)
    assert not oracle.theta_weak((0, 0), 2.0, (4.0, 0), 0.5, 0.25)
    # a point-like leaf next to a large one: apart is enough for the exchange, touching is not
    assert oracle.theta_swapped((0, 0), 1.0, (1.5, 0), 0.0, 0.5)
    assert not oracle.theta_swapped((0, 0), 1.0, (1.0, 0), 0.0, 0.5)


def test_swapped_criterion_is_the_small_set_expanded():
    # the exchanged test asks that the smaller set, expanded by 1/theta about its centre, stay
    # clear of the larger one: r/theta + R < d (r <= R); with equal radii it is Criterion 2.1,
    # and whatever Criterion 2.1 accepts it accepts too
    g = np.random.default_rng(5)
    for _ in range(4000):
        th = g.uniform(0.05, 0.95)
        r1, r2 = g.uniform(0, 1, 2)
        c1, c2 = g.uniform(-4, 4, 2), g.uniform(-4, 4, 2)
        d = np.hypot(*(c1 - c2))
        R, r = max(r1, r2), min(r1, r2)
        margin = d - (r / th + R)
        if abs(margin) < 1e-9:
            continue
        sw = oracle.theta_swapped(c1, r1, c2, r2, th)
        assert sw == (margin > 0)
        assert sw == oracle.theta_swapped(c2, r2, c1, r1, th)
        if oracle.theta_weak(c1, r1, c2, r2, th):
            assert sw
        assert oracle.theta_swapped(c1, r1, c2, r1, th) == oracle.theta_weak(c1, r1, c2, r1, th)


@pytest.mark.parametrize("p", [4, 8, 16, 30])
def test_p2l_within_series_bound(p):
    src, tgt, q = _disc_and_annulus(1)
    c = 0.02 - 0.01j  # an off-origin centre
    b = oracle.p2l(src.real, src.imag, q, (c.real, c.imag), p)
    ratio = np.max(np.abs(tgt - c)) / np.min(np.abs(src - c))
    bound = np.sum(np.abs(q)) * ratio ** (p + 1) / ((p + 1) * (1 - ratio))
    for z in tgt:
        got = oracle.l2p(b, z - c, p)
        ref = np.sum(q * np.log(np.abs(z - src)))
        assert abs(got - ref) <= bound * (1 + 1e-9) + 1e-13 * np.sum(np.abs(q))


def test_p2l_high_order_is_direct():
    src, tgt, q = _disc_and_annulus(2)
    b = oracle.p2l(src.real, src.imag, q, (0.0, 0.0), 40)
    for z in tgt:
        ref = np.sum(q * np.log(np.abs(z - src)))
        assert abs(oracle.l2p(b, z, 40) - ref) <= 1e-13 * np.sum(np.abs(q))


@pytest.mark.parametrize("p", [4, 8, 16, 30])
def test_m2p_within_series_bound(p):
    # the same geometry seen the other way: sources in the small disc, targets in the annulus
    tgt, src, q = _disc_and_annulus(3, m_src=25, m_tgt=40)
    q = np.random.default_rng(4).normal(size=src.shape[0])
    c = -0.01 + 0.03j
    a = oracle.p2m(src.real, src.imag, q, (c.real, c.imag), p)
    ratio = np.max(np.abs(src - c)) / np.min(np.abs(tgt - c))
    bound = np.sum(np.abs(q)) * ratio ** (p + 1) / ((p + 1) * (1 - ratio))
    for z in tgt:
        got = oracle.m2p(a, z - c, p)
        ref = np.sum(q * np.log(np.abs(z - src)))
        assert abs(got - ref) <= bound * (1 + 1e-9) + 1e-13 * np.sum(np.abs(q))


CLOUDS = [
    ("clusters", lambda: W.clusters(20000, 71), 5),
    ("rings", lambda: W.rings_plummer(16384, 72), 5),
    ("uniform", lambda: W.uniform(9000, 73), 4),
]


@pytest.mark.parametrize("theta", [0.5, 0.35])
@pytest.mark.parametrize("k", range(len(CLOUDS)))
def test_exchange_lists_split_the_strong_lists(k, theta):
    _, make, L = CLOUDS[k]
    c = make()
    perm, rects, lb = oracle.tree(c.x, c.y, L)
    pw, pi, ps, psi = oracle.lists(rects, L, theta)
    w, wi, s, si, xo, xi = oracle.lists(rects, L, theta, swap=True)
    assert np.array_equal(pw, w) and np.array_equal(pi, wi)  # weak lists untouched
    base = (4 ** L - 1) // 3
    assert np.array_equal(ps[:base + 1], s[:base + 1]) and np.all(xo[:base + 1] == 0)
    cen, rad = oracle.geometry(rects)
    z = (c.x + 1j * c.y)[perm]
    nx = 0
    for b in range(4 ** L):
        g = base + b
        plain = psi[ps[g]:ps[g + 1]]
        kept = si[s[g]:s[g + 1]]
        ex = xi[xo[g]:xo[g + 1]]
        src = ex & ~oracle.SWAP_M2P
        # an order-preserving split of the plain list
        is_x = np.isin(plain, src)
        assert np.array_equal(plain[~is_x], kept) and np.array_equal(plain[is_x], src)
        for v, m2p in zip(src, (ex & oracle.SWAP_M2P) != 0):
            sg = base + v
            zt, zs = z[lb[b]:lb[b + 1]], z[lb[v]:lb[v + 1]]
            ct, cs = cen[g, 0] + 1j * cen[g, 1], cen[sg, 0] + 1j * cen[sg, 1]
            assert rad[g] != rad[sg] and m2p == (rad[g] > rad[sg])
            if m2p:   # source expansion about cs, evaluated at the target's points
                assert np.max(np.abs(zs - cs)) <= theta * np.min(np.abs(zt - cs)) * (1 + 1e-12)
            else:     # local expansion about ct of the source's points
                assert np.max(np.abs(zt - ct)) <= theta * np.min(np.abs(zs - ct)) * (1 + 1e-12)
        nx += ex.size
    if CLOUDS[k][0] != "uniform":
        assert nx > 0


def test_lattice_exchanges_only_border_leaves():
    # a 64 x 64 lattice: interior leaves of a 4-level tree are congruent 4 x 4 blocks; the leaves
    # on the border are half a spacing narrower (the root is the points' bounding box), so only
    # pairs of leaves of different shapes, one of them on the border, can be exchanged
    g = np.arange(64) + 0.5
    X, Y = np.meshgrid(g, g, indexing="ij")
    x, y = X.ravel() / 64, Y.ravel() / 64
    _, rects, _ = oracle.tree(x, y, 4)
    _, _, _, _, xo, xi = oracle.lists(rects, 4, 0.5, swap=True)
    base = (4 ** 4 - 1) // 3
    lo, hi = rects[:, [0, 2]].min(), rects[:, [1, 3]].max()
    border = (np.isclose(rects[:, [0, 2]], lo).any(axis=1)) | (np.isclose(rects[:, [1, 3]], hi).any(axis=1))
    assert xo[-1] > 0
    shape = np.round((rects[:, [1, 3]] - rects[:, [0, 2]]) * 128).astype(int)  # in half spacings
    for b in range(4 ** 4):
        for v in xi[xo[base + b]:xo[base + b + 1]] & ~oracle.SWAP_M2P:
            assert border[base + b] or border[base + v]
            assert not np.array_equal(shape[base + b], shape[base + v])


@pytest.mark.parametrize("L", [0, 1])
def test_touching_leaves_exchange_nothing(L):
    c = W.clusters(3000, 76)
    _, rects, _ = oracle.tree(c.x, c.y, L)
    assert oracle.lists(rects, L, 0.5, swap=True)[4][-1] == 0
    assert np.array_equal(oracle.fmm(c.x, c.y, c.q, L, 10, 0.5, swap=True), oracle.fmm(c.x, c.y, c.q, L, 10, 0.5))


@pytest.mark.parametrize("parents", [False, True])
def test_method_with_exchange_converges(parents):
    c = W.clusters(8000, 74)
    d = oracle.direct(c.x, c.y, c.q)
    errs = []
    for p in (4, 8, 12, 16):
        f = oracle.fmm(c.x, c.y, c.q, 5, p, 0.5, parents=parents, swap=True)
        errs.append(np.max(np.abs(f - d)) / np.max(np.abs(d)))
    errs = np.array(errs)
    assert np.all(errs[1:] <= errs[:-1] / 8)
    assert np.all(errs <= 0.5 ** (np.array([4, 8, 12, 16]) + 1) / 0.25)


def test_field_with_exchange_converges():
    c = W.clusters(6000, 75)
    d = oracle.direct_field(c.x, c.y, c.q)
    errs = []
    for p in (4, 8, 12, 16):
        f = oracle.fmm_field(c.x, c.y, c.q, 5, p, 0.5, swap=True)
        errs.append(np.max(np.abs(f - d)) / np.max(np.abs(d)))
    errs = np.array(errs)
    assert np.all(errs[1:] <= errs[:-1] / 8)
    assert np.all(errs <= 0.5 ** (np.array([4, 8, 12, 16]) + 1) / 0.25)
