"""Pins for the CPU oracle: it is checked against what the paper and the mathematics fix --
closed forms, textbook error bounds, exact identities, invariants and brute force on tiny
inputs -- never against itself.  CPU only."""
import math

import numpy as np
import pytest

from paper_1006_2269_gb300 import workloads as W


# ---------------------------------------------------------------------------------------------
# Eq. (1.1), direct summation
# ---------------------------------------------------------------------------------------------

def test_direct_two_points(orc):
    # Phi_0 = q_1 log d, Phi_1 = q_0 log d
    x = np.array([0.25, 0.25 + 3.0])
    y = np.array([-1.0, -1.0 + 4.0])
    q = np.array([2.0, -0.5])
    phi = orc.direct(x, y, q)
    assert phi[0] == pytest.approx(-0.5 * math.log(5.0), rel=1e-15)
    assert phi[1] == pytest.approx(2.0 * math.log(5.0), rel=1e-15)


@pytest.mark.parametrize("n,R", [(7, 1.0), (64, 0.3), (257, 2.5)])
def test_direct_roots_of_unity(orc, n, R):
    # prod_{j != i} |z_i - z_j| = n R^(n-1) for n equally spaced points on a circle of radius R
    t = 2 * np.pi * np.arange(n) / n
    x, y = 0.1 + R * np.cos(t), -0.2 + R * np.sin(t)
    phi = orc.direct(x, y, np.ones(n))
    assert np.allclose(phi, math.log(n) + (n - 1) * math.log(R), rtol=0, atol=1e-11 * n)


def test_direct_skips_coincident(orc):
    # reading R7: a coincident distinct point contributes nothing
    x = np.array([0.0, 0.0, 1.0])
    y = np.array([0.0, 0.0, 0.0])
    q = np.array([1.0, 5.0, 3.0])
    phi = orc.direct(x, y, q)
    assert phi[0] == 0.0 and phi[1] == 0.0  # log 1 = 0 from the third point
    assert phi[2] == 0.0


# ---------------------------------------------------------------------------------------------
# Criterion 2.1
# ---------------------------------------------------------------------------------------------

def test_theta_criterion_hand_values(orc):
    # r1 = r2 = 1, theta = 1/2: well separated iff 1 + 0.5 <= 0.5 d, i.e. d >= 3
    assert orc.theta_weak((0, 0), 1.0, (3.0, 0), 1.0, 0.5)
    assert not orc.theta_weak((0, 0), 1.0, (2.9999999, 0), 1.0, 0.5)
    # R = 2, r = 0.5, theta = 1/4: 2 + 0.125 <= 0.25 d  <=>  d >= 8.5
    assert orc.theta_weak((0, 0), 2.0, (0.0, 8.5), 0.5, 0.25)
    assert not orc.theta_weak((0, 0), 2.0, (0.0, 8.49), 0.5, 0.25)
    assert not orc.theta_weak((0, 0), 2.0, (6.0, 6.0), 0.5, 0.25)  # d = 8.485...
    # two point-like boxes: well separated when apart, never when they coincide (reading R5)
    assert orc.theta_weak((0, 0), 0.0, (1e-3, 0), 0.0, 0.5)
    assert not orc.theta_weak((0, 0), 0.0, (0, 0), 0.0, 0.5)


def test_theta_criterion_is_expand_and_rotate(orc):
    # Paper, after Criterion 2.1: well separated iff either set can be expanded by 1/theta about
    # its centre without touching the other, i.e. R/theta + r <= d; and the criterion is symmetric.
    g = np.random.default_rng(1)
    for _ in range(4000):
        th = g.uniform(0.05, 0.95)
        r1, r2 = g.uniform(0, 1, 2)
        c1, c2 = g.uniform(-5, 5, 2), g.uniform(-5, 5, 2)
        d = np.hypot(*(c1 - c2))
        R, r = max(r1, r2), min(r1, r2)
        margin = d - (R / th + r)
        if abs(margin) < 1e-9:
            continue
        w = orc.theta_weak(c1, r1, c2, r2, th)
        assert w == (margin > 0)
        assert w == orc.theta_weak(c2, r2, c1, r1, th)


# ---------------------------------------------------------------------------------------------
# Tree (Section 4, Fig. 1.1, Fig. 4.1): checked against an independent characterisation
# ---------------------------------------------------------------------------------------------

def check_tree(x, y, L, perm, rects, lb):
    n = x.shape[0]
    assert np.array_equal(np.sort(perm), np.arange(n))
    nleaf = 4 ** L
    assert lb[0] == 0 and lb[-1] == n and np.all(np.diff(lb) >= 1)
    assert np.array_equal(rects[0], [x.min(), x.max(), y.min(), y.max()])
    # inside each leaf: ascending input index (reading R8)
    for b in range(nleaf):
        s = perm[lb[b]:lb[b + 1]]
        assert np.all(np.diff(s) > 0)

    def pts(l, b):
        s = 4 ** (L - l)
        return perm[lb[b * s]:lb[(b + 1) * s]]

    def lexmax(c, ids):
        k = np.lexsort((ids, c[ids]))
        return c[ids[k[-1]]], ids[k[-1]]

    def lexmin(c, ids):
        k = np.lexsort((ids, c[ids]))
        return c[ids[k[0]]], ids[k[0]]

    for l in range(L + 1):
        nb = 4 ** l
        base = (4 ** l - 1) // 3
        for b in range(nb):
            P = pts(l, b)
            m = P.shape[0]
            assert m in (n // nb, -(-n // nb))  # balanced tree: floor or ceil of N / 4^l
            r = rects[base + b]
            assert np.all((x[P] >= r[0]) & (x[P] <= r[1]) & (y[P] >= r[2]) & (y[P] <= r[3]))
            if l == L:
                continue
            ch = [pts(l + 1, 4 * b + k) for k in range(4)]
            xlo, xhi = np.concatenate(ch[:2]), np.concatenate(ch[2:])
            assert xlo.shape[0] == m // 2  # lower x-half gets floor(m/2) (reading R1)
            a, ai = lexmax(x, xlo)
            c, ci = lexmin(x, xhi)
            assert (a, ai) < (c, ci)  # median split in (x, index) order (reading R2)
            xs = 0.5 * (a + c)  # reading R3
            ys = []
            for lo, hi in ((ch[0], ch[1]), (ch[2], ch[3])):
                assert lo.shape[0] == (lo.shape[0] + hi.shape[0]) // 2
                a2, a2i = lexmax(y, lo)
                c2, c2i = lexmin(y, hi)
                assert (a2, a2i) < (c2, c2i)
                ys.append(0.5 * (a2 + c2))
            cb = (4 ** (l + 1) - 1) // 3 + 4 * b
            want = np.array([[r[0], xs, r[2], ys[0]], [r[0], xs, ys[0], r[3]],
                             [xs, r[1], r[2], ys[1]], [xs, r[1], ys[1], r[3]]])
            assert np.array_equal(rects[cb:cb + 4], want)


def test_tree_hand_example(orc):
    # unit-square corners with L = 1: x-split at 0.5 takes inputs {0, 2}; each half splits at
    # y = 0.5; children in id order (xl,yl), (xl,yh), (xh,yl), (xh,yh).
    x = np.array([0.0, 1.0, 0.0, 1.0])
    y = np.array([0.0, 0.0, 1.0, 1.0])
    perm, rects, lb = orc.tree(x, y, 1)
    assert perm.tolist() == [0, 2, 1, 3]
    assert lb.tolist() == [0, 1, 2, 3, 4]
    assert rects.tolist() == [[0, 1, 0, 1], [0, .5, 0, .5], [0, .5, .5, 1],
                              [.5, 1, 0, .5], [.5, 1, .5, 1]]


def test_tree_ties_by_index(orc):
    # five points on one vertical line: x ties are broken by input index (reading R2)
    x = np.zeros(5)
    y = np.array([4.0, 3.0, 2.0, 1.0, 0.0])
    perm, rects, lb = orc.tree(x, y, 1)
    # x-low = inputs {0, 1}; split of {0,1} by y: y-low {1} ; x-high {2,3,4}: y-low {4}
    assert lb.tolist() == [0, 1, 2, 3, 5]
    assert perm.tolist() == [1, 0, 4, 2, 3]
    assert rects[1].tolist() == [0, 0, 0, 3.5]  # zero-width box, ys = 0.5*(3+4)
    check_tree(x, y, 1, perm, rects, lb)


CASES = [
    ("uniform", lambda: W.uniform(1000, 1), 2),
    ("ragged", lambda: W.uniform(4 ** 3 + 13, 2), 3),
    ("exact", lambda: W.uniform(4 ** 4, 3), 4),
    ("clusters", lambda: W.clusters(3001, 4), 3),
    ("circle", lambda: W.circle(777, 5), 3),
    ("normal", lambda: W.normal(555, 6), 2),
    ("rings", lambda: W.rings_plummer(2000, 7), 3),
]


def _dupes():
    c = W.uniform(400, 8)
    x = np.round(c.x * 8) / 8  # many exact duplicates and collinear rows
    y = np.round(c.y * 8) / 8
    return W.Cloud(x, y, c.q, "dupes")


CASES.append(("dupes", _dupes, 3))


@pytest.mark.parametrize("name,make,L", CASES, ids=[c[0] for c in CASES])
def test_tree_invariants(orc, name, make, L):
    c = make()
    perm, rects, lb = orc.tree(c.x, c.y, L)
    check_tree(c.x, c.y, L, perm, rects, lb)


def test_tree_rejects_too_few_points(orc):
    with pytest.raises(orc.OracleError):
        orc.tree(np.zeros(15), np.zeros(15), 2)


# ---------------------------------------------------------------------------------------------
# Box geometry (reading R4: the sphere of Criterion 2.1 is the circumscribed circle of the
# partition rectangle, so centre = midpoint and radius = half the diagonal)
# ---------------------------------------------------------------------------------------------

@pytest.mark.parametrize("rect,centre,radius", [
    ((0.0, 1.0, 0.0, 1.0), (0.5, 0.5), math.sqrt(2.0) / 2),    # unit square
    ((0.0, 2.0, 0.0, 1.0), (1.0, 0.5), math.sqrt(5.0) / 2),    # 2 x 1 rectangle
    ((-3.0, 1.0, 2.0, 5.0), (-1.0, 3.5), 2.5),                  # 4 x 3: a 3-4-5 diagonal
    ((3.0, 3.0, 1.0, 5.0), (3.0, 3.0), 2.0),                    # zero width: a segment
    ((0.25, 0.25, -0.5, -0.5), (0.25, -0.5), 0.0),              # a point box
], ids=["unit", "2x1", "3-4-5", "zero-width", "point"])
def test_geometry_hand_values(orc, rect, centre, radius):
    cen, rad = orc.geometry(np.array([rect], dtype=np.float64))
    assert cen[0].tolist() == pytest.approx(list(centre), rel=0, abs=1e-15)
    assert rad[0] == pytest.approx(radius, rel=1e-15, abs=0)


def test_geometry_is_the_smallest_enclosing_circle(orc):
    # The circle through the four corners about the midpoint is the smallest disc holding the
    # rectangle: every corner lies on it (a larger radius, e.g. the whole diagonal, fails), and
    # two opposite corners are a diameter apart (a smaller one cannot hold both).
    rng = np.random.default_rng(424242)
    lo = rng.uniform(-5, 5, (200, 2))
    ext = rng.uniform(0, 3, (200, 2)) * (rng.uniform(size=(200, 2)) > 0.1)
    rects = np.stack([lo[:, 0], lo[:, 0] + ext[:, 0], lo[:, 1], lo[:, 1] + ext[:, 1]], axis=1)
    cen, rad = orc.geometry(rects)
    for (x0, x1, y0, y1), c, r in zip(rects, cen, rad):
        for cx_, cy_ in ((x0, y0), (x0, y1), (x1, y0), (x1, y1)):
            assert math.hypot(cx_ - c[0], cy_ - c[1]) == pytest.approx(r, rel=1e-14, abs=1e-300)
        assert 2 * r == pytest.approx(math.hypot(x1 - x0, y1 - y0), rel=1e-15, abs=1e-300)


# ---------------------------------------------------------------------------------------------
# Connectivity (Section 4)
# ---------------------------------------------------------------------------------------------

def brute_lists(orc, rects, L, theta):
    """All same-level pairs, level by level: (b, c) is examined iff their parents are strongly
    coupled; then weak iff the criterion holds."""
    cen, rad = orc.geometry(rects)
    strong_prev = {(0, 0)}
    out = {0: ({0: []}, {0: [0]})}
    for l in range(1, L + 1):
        base = (4 ** l - 1) // 3
        nb = 4 ** l
        Wl = {b: [] for b in range(nb)}
        Sl = {b: [] for b in range(nb)}
        for b in range(nb):
            for c in range(nb):
                if (b // 4, c // 4) not in strong_prev:
                    continue
                w = orc.theta_weak(cen[base + b], rad[base + b], cen[base + c], rad[base + c], theta)
                (Wl if w else Sl)[b].append(c)
        strong_prev = {(b, c) for b in range(nb) for c in Sl[b]}
        out[l] = (Wl, Sl)
    return out


@pytest.mark.parametrize("theta", [0.25, 0.5, math.sqrt(0.5)])
@pytest.mark.parametrize("name,make,L", [CASES[0], CASES[3], CASES[4], CASES[-1]],
                         ids=["uniform", "clusters", "circle", "dupes"])
def test_lists_brute_force(orc, name, make, L, theta):
    c = make()
    perm, rects, lb = orc.tree(c.x, c.y, L)
    woff, widx, soff, sidx = orc.lists(rects, L, theta)
    ref = brute_lists(orc, rects, L, theta)
    for l in range(L + 1):
        base = (4 ** l - 1) // 3
        for b in range(4 ** l):
            g = base + b
            assert widx[woff[g]:woff[g + 1]].tolist() == ref[l][0][b]
            assert sidx[soff[g]:soff[g + 1]].tolist() == ref[l][1][b]
            assert b in sidx[soff[g]:soff[g + 1]]  # a box is strongly coupled to itself


def brute_lists_own_geometry(rects, L, theta):
    """The same brute force with nothing taken from the oracle: circumscribed circles and
    Criterion 2.1 written out here, in the arithmetic order of their definitions."""
    rects = np.asarray(rects, dtype=np.float64)
    cen = [(0.5 * (r[0] + r[1]), 0.5 * (r[2] + r[3])) for r in rects]
    rad = [0.5 * math.sqrt((r[1] - r[0]) * (r[1] - r[0]) + (r[3] - r[2]) * (r[3] - r[2])) for r in rects]

    def weak(a, b):
        dx, dy = cen[a][0] - cen[b][0], cen[a][1] - cen[b][1]
        d = math.sqrt(dx * dx + dy * dy)
        R, r = max(rad[a], rad[b]), min(rad[a], rad[b])
        return R + theta * r <= theta * d and R + r < d

    strong_prev = {(0, 0)}
    out = {}
    for l in range(1, L + 1):
        base = (4 ** l - 1) // 3
        Wl, Sl = {}, {}
        for b in range(4 ** l):
            cand = [c for c in range(4 ** l) if (b // 4, c // 4) in strong_prev]
            Wl[b] = [c for c in cand if weak(base + b, base + c)]
            Sl[b] = [c for c in cand if not weak(base + b, base + c)]
        strong_prev = {(b, c) for b in Sl for c in Sl[b]}
        out[l] = (Wl, Sl)
    return out


@pytest.mark.parametrize("theta", [0.25, 0.5, math.sqrt(0.5)])
@pytest.mark.parametrize("name,make,L", [CASES[0], CASES[3]], ids=["uniform", "clusters"])
def test_lists_brute_force_own_geometry(orc, name, make, L, theta):
    c = make()
    perm, rects, lb = orc.tree(c.x, c.y, L)
    woff, widx, soff, sidx = orc.lists(rects, L, theta)
    ref = brute_lists_own_geometry(rects, L, theta)
    for l in range(1, L + 1):
        base = (4 ** l - 1) // 3
        for b in range(4 ** l):
            g = base + b
            assert widx[woff[g]:woff[g + 1]].tolist() == ref[l][0][b]
            assert sidx[soff[g]:soff[g + 1]].tolist() == ref[l][1][b]


@pytest.mark.parametrize("theta", [0.25, 0.5, math.sqrt(0.5)])
def test_lists_symmetry_and_inequalities(orc, theta):
    c = W.clusters(5000, 11)
    L = 4
    perm, rects, lb = orc.tree(c.x, c.y, L)
    cen, rad = orc.geometry(rects)
    woff, widx, soff, sidx = orc.lists(rects, L, theta)
    for l in range(1, L + 1):
        base = (4 ** l - 1) // 3
        Wset = {(b, int(v)) for b in range(4 ** l) for v in widx[woff[base + b]:woff[base + b + 1]]}
        Sset = {(b, int(v)) for b in range(4 ** l) for v in sidx[soff[base + b]:soff[base + b + 1]]}
        assert all((v, b) in Wset for (b, v) in Wset)  # the criterion is symmetric (Section 2)
        assert all((v, b) in Sset for (b, v) in Sset)
        for (b, v) in Wset:
            d = np.hypot(*(cen[base + b] - cen[base + v]))
            R, r = max(rad[base + b], rad[base + v]), min(rad[base + b], rad[base + v])
            # Eqs. (2.1) and (2.2), consequences of the criterion
            assert (d + r + R) / (d - R) <= 2 / (1 - theta) * (1 + 1e-12)
            assert r / (d - R) <= R / (d - r) * (1 + 1e-12) + 1e-300
            assert R / (d - r) <= theta * (1 + 1e-12)


@pytest.mark.parametrize("theta", [0.25, 0.5, math.sqrt(0.5)])
@pytest.mark.parametrize("name,make,L", [CASES[0], CASES[1], CASES[3], CASES[-1]],
                         ids=["uniform", "ragged", "clusters", "dupes"])
def test_lists_partition_of_interactions(orc, name, make, L, theta):
    # every ordered pair i != j is handled exactly once: by M2L on exactly one level, or by the
    # direct sum along the finest strong lists
    c = make()
    n = c.x.shape[0]
    if n > 3100:
        pytest.skip("brute force too large")
    perm, rects, lb = orc.tree(c.x, c.y, L)
    woff, widx, soff, sidx = orc.lists(rects, L, theta)
    leaf = np.empty(n, np.int64)
    for b in range(4 ** L):
        leaf[perm[lb[b]:lb[b + 1]]] = b
    count = np.zeros((n, n), np.int32)
    for l in range(1, L + 1):
        base = (4 ** l - 1) // 3
        nb = 4 ** l
        Wm = np.zeros((nb, nb), bool)
        for b in range(nb):
            Wm[b, widx[woff[base + b]:woff[base + b + 1]]] = True
        anc = leaf >> (2 * (L - l))
        count += Wm[anc[:, None], anc[None, :]]
    base = (4 ** L - 1) // 3
    Sm = np.zeros((4 ** L, 4 ** L), bool)
    for b in range(4 ** L):
        Sm[b, sidx[soff[base + b]:soff[base + b + 1]]] = True
    count += Sm[leaf[:, None], leaf[None, :]]
    np.fill_diagonal(count, 1)
    assert np.all(count == 1)


# ---------------------------------------------------------------------------------------------
# Expansion operators (classical complex representation, Section 5 / ref. [FMM])
# ---------------------------------------------------------------------------------------------

def _cluster(g, m, c, r):
    t = g.uniform(0, 2 * np.pi, m)
    s = r * np.sqrt(g.random(m))
    return c[0] + s * np.cos(t), c[1] + s * np.sin(t), g.uniform(-1, 1, m)


@pytest.mark.parametrize("p", [2, 5, 10, 20, 30])
def test_multipole_truncation_bound(orc, p):
    # textbook bound: |phi - M2P| <= A/(p+1) * a^(p+1) / (1 - a), a = r/|z - c|, A = sum |q|
    g = np.random.default_rng(p)
    c = np.array([0.3, -0.2])
    r = 0.5
    xs, ys, q = _cluster(g, 60, c, r)
    a = orc.p2m(xs, ys, q, c, p)
    A = np.abs(q).sum()
    for _ in range(20):
        ang = g.uniform(0, 2 * np.pi)
        R = g.uniform(1.2, 4.0) * r
        z = c + R * np.array([np.cos(ang), np.sin(ang)])
        exact = np.sum(q * np.log(np.hypot(z[0] - xs, z[1] - ys)))
        approx = orc.m2p(a, complex(*(z - c)), p)
        al = r / R
        assert abs(exact - approx) <= A / (p + 1) * al ** (p + 1) / (1 - al) * (1 + 1e-9) + 1e-13 * A


@pytest.mark.parametrize("p", [3, 12, 25])
def test_m2m_is_exact(orc, p):
    # shifting a p-term multipole loses nothing: P2M about the parent centre equals M2M of the
    # children's multipoles, coefficient by coefficient
    g = np.random.default_rng(100 + p)
    cp = np.array([0.5, 0.5])
    tot = np.zeros(p + 1, complex)
    X, Y, Q = [], [], []
    for k in range(4):
        cc = cp + g.uniform(-0.25, 0.25, 2)
        xs, ys, q = _cluster(g, 17, cc, 0.1)
        X.append(xs), Y.append(ys), Q.append(q)
        tot += orc.m2m(orc.p2m(xs, ys, q, cc, p), complex(*(cc - cp)), p)
    direct = orc.p2m(np.concatenate(X), np.concatenate(Y), np.concatenate(Q), cp, p)
    scale = np.abs(direct).max()
    assert np.allclose(tot, direct, rtol=0, atol=1e-13 * scale)


@pytest.mark.parametrize("p", [3, 12, 25])
def test_l2l_is_polynomial_recentring(orc, p):
    g = np.random.default_rng(200 + p)
    b = g.standard_normal(p + 1) + 1j * g.standard_normal(p + 1)
    z0 = complex(*g.uniform(-0.3, 0.3, 2))
    bc = orc.l2l(b, z0, p)
    for _ in range(10):
        w = complex(*g.uniform(-0.3, 0.3, 2))
        assert orc.l2p(bc, w, p) == pytest.approx(orc.l2p(b, w + z0, p), rel=1e-12, abs=1e-12)


@pytest.mark.parametrize("theta", [0.25, 0.5, math.sqrt(0.5)])
def test_m2l_single_pair_error_decay(orc, theta):
    # two sets satisfying Criterion 2.1 at equality; the local expansion obtained by
    # P2M -> M2L must reproduce the potential with an error falling like theta^(p+1)
    # (Section 3: relative error <= const * theta^(p+1) / (1-theta)^2).
    g = np.random.default_rng(7)
    rs, rt = 0.2, 0.13
    R, r = max(rs, rt), min(rs, rt)
    d = (R + theta * r) / theta
    cs, ct = np.array([0.0, 0.0]), np.array([d * 0.6, d * 0.8])
    xs, ys, q = _cluster(g, 80, cs, rs)
    xt, yt, _ = _cluster(g, 40, ct, rt)
    A = np.abs(q).sum()
    exact = np.array([np.sum(q * np.log(np.hypot(a - xs, b - ys))) for a, b in zip(xt, yt)])
    prev = np.inf
    for p in range(2, 40, 3):
        loc = orc.m2l(orc.p2m(xs, ys, q, cs, p), complex(*(cs - ct)), p)
        approx = np.array([orc.l2p(loc, complex(a - ct[0], b - ct[1]), p) for a, b in zip(xt, yt)])
        err = np.abs(approx - exact).max() / A
        assert err <= 4 * (p + 1) * theta ** (p + 1) / (1 - theta) ** 2 + 1e-14
        assert err <= prev * 1.05 + 1e-14
        prev = err


def test_m2l_single_source_closed_form(orc):
    # one unit source at s, local expansion about 0: b_0 = log|s| (real part), b_l = -1/(l s^l)
    # (log(z - s) = log(-s) - sum_l (z/s)^l / l)
    s = complex(3.0, -4.0)
    p = 12
    a = orc.p2m(np.array([3.0]), np.array([-4.0]), np.array([1.0]), (3.0, -4.0), p)
    assert a[0] == 1.0 and np.all(a[1:] == 0)  # multipole about the source itself
    loc = orc.m2l(a, s, p)
    assert loc[0].real == pytest.approx(math.log(5.0), rel=1e-15)
    for l in range(1, p + 1):
        assert loc[l] == pytest.approx(-1.0 / (l * s ** l), rel=1e-13)


# ---------------------------------------------------------------------------------------------
# The whole method
# ---------------------------------------------------------------------------------------------

def test_fmm_L0_is_direct(orc):
    c = W.uniform(300, 21)
    assert np.allclose(orc.fmm(c.x, c.y, c.q, 0, 10, 0.5), orc.direct(c.x, c.y, c.q), rtol=0, atol=1e-13)


def test_fmm_without_weak_pairs_is_direct(orc):
    # L = 1 on uniform points: the four children of the root touch, so no pair is weak and the
    # method reduces to the direct sum
    c = W.uniform(2000, 22)
    perm, rects, lb = orc.tree(c.x, c.y, 1)
    woff, widx, soff, sidx = orc.lists(rects, 1, 0.5)
    assert widx.shape[0] == 0
    ref = orc.direct(c.x, c.y, c.q)
    assert np.allclose(orc.fmm(c.x, c.y, c.q, 1, 5, 0.5), ref, rtol=0, atol=1e-12 * np.abs(ref).max())


@pytest.mark.parametrize("n,R", [(1024, 1.0), (3000, 0.5)])
def test_fmm_roots_of_unity(orc, n, R):
    t = 2 * np.pi * np.arange(n) / n
    x, y = 0.5 + R * np.cos(t), 0.5 + R * np.sin(t)
    phi = orc.fmm(x, y, np.ones(n), 3, 20, 0.5)
    want = math.log(n) + (n - 1) * math.log(R)
    assert np.abs(phi - want).max() <= 1e-6 * max(abs(want), 1.0) * n


@pytest.fixture(scope="module")
def sweep(orc):
    c = W.uniform(4096, 23)
    ref = orc.direct(c.x, c.y, c.q, nthreads=4)
    out = {}
    for th in (0.25, 0.5, math.sqrt(0.5)):
        for p in range(2, 32, 2):
            phi = orc.fmm(c.x, c.y, c.q, 3, p, th)
            out[(th, p)] = np.abs(phi - ref).max() / np.abs(ref).max()
    return out


def test_error_bound_theta_p(sweep):
    # Section 3: relative error <= const * theta^(p+1) / (1-theta)^2, one constant for all
    for (th, p), e in sweep.items():
        assert e <= 1.0 * th ** (p + 1) / (1 - th) ** 2 + 5e-14


def test_error_monotone_in_p_and_theta(sweep):
    for th in (0.25, 0.5, math.sqrt(0.5)):
        errs = [sweep[(th, p)] for p in range(2, 32, 2)]
        for a, b in zip(errs, errs[1:]):
            assert b <= a * 1.05 + 2e-14  # non-increasing down to the FP64 floor
        ps = np.arange(2, 32, 2)
        e = np.array(errs)
        m = e > 1e-12
        slope = np.polyfit(ps[m], np.log(e[m]), 1)[0]
        # geometric decay at least as fast as the estimate's theta^(p+1)
        assert 3.0 * math.log(th) < slope < 0.9 * math.log(th)
    for p in range(2, 20, 2):  # smaller theta, smaller error (Section 2, after Criterion 2.1)
        assert sweep[(0.25, p)] <= sweep[(0.5, p)] <= sweep[(math.sqrt(0.5), p)]


def test_p20_reaches_1e6(orc):
    # Section 5: p = 20 with theta = 1/2 gives a relative tolerance of about 1e-6
    c = W.plain_fp64_cloud()
    phi = orc.fmm(c.x, c.y, c.q, 4, 20, 0.5)
    ref = orc.direct(c.x, c.y, c.q, nthreads=4)
    assert np.abs(phi - ref).max() / np.abs(ref).max() <= 1e-6


def test_coefficients_consistent_with_p2m(orc):
    # the multipole of every box after the upward pass is P2M of all its points (M2M is exact)
    c = W.clusters(2000, 24)
    L, p = 3, 9
    phi, M, Lc = orc.fmm(c.x, c.y, c.q, L, p, 0.5, want_coeffs=True)
    perm, rects, lb = orc.tree(c.x, c.y, L)
    cen, rad = orc.geometry(rects)
    for l in range(L + 1):
        base = (4 ** l - 1) // 3
        s = 4 ** (L - l)
        for b in range(4 ** l):
            P = perm[lb[b * s]:lb[(b + 1) * s]]
            a = orc.p2m(c.x[P], c.y[P], c.q[P], cen[base + b], p)
            scale = np.abs(c.q[P]).sum() * np.maximum(rad[base + b], 1e-300) ** np.arange(p + 1)
            assert np.all(np.abs(M[base + b] - a) <= 1e-12 * scale + 1e-300)
