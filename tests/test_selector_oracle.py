"""Pins of the FP64 selector reference (oracle/mlp_oracle.c), all on the CPU.

The network reference is pinned by central finite differences of its own loss (gradient), by
closed forms (zero parameters; an output layer of biases only), and by a hand-wired network whose
output is known in advance (identity paths through the ReLU layers), so that a transposed weight,
a dropped bias or a wrong ReLU derivative fails a test.  The features are pinned on hand-built
partition rectangles whose statistics are known exactly.
"""
import math

import numpy as np
import pytest

import oracle
from oracle import mlp as M

NI, NH, NO = 64, 128, 225
O_W1, O_B1 = 0, NH * NI
O_W2, O_B2 = O_B1 + NH, O_B1 + NH + NH * NH
O_W3, O_B3 = O_B2 + NH, O_B2 + NH + NO * NH


def test_parameter_count():
    assert M.nparams() == 53857 == O_B3 + NO


def _softmax(z):
    e = np.exp(z - z.max(axis=-1, keepdims=True))
    return e / e.sum(axis=-1, keepdims=True)


def test_zero_parameters_closed_form():
    X = np.random.default_rng(1).normal(size=(6, NI))
    y = np.array([0, 5, 224, 17, 17, 100])
    p = np.zeros(M.nparams())
    prob = M.forward(p, X)
    assert np.allclose(prob, 1.0 / NO, rtol=0, atol=1e-15)
    loss, g = M.loss_grad(p, X, y)
    assert abs(loss - math.log(NO)) < 1e-13
    gb3 = np.full(NO, 1.0 / NO)
    for v in y:
        gb3[v] -= 1.0 / len(y)
    assert np.allclose(g[O_B3:], gb3, atol=1e-15)
    assert np.all(g[:O_B3] == 0.0)  # hidden activations are 0, so nothing else moves


def test_bias_only_output_layer():
    rng = np.random.default_rng(2)
    p = rng.normal(0, 0.3, M.nparams())
    p[O_W3:O_B3] = 0.0
    b3 = p[O_B3:].copy()
    X = rng.normal(size=(4, NI))
    y = np.array([3, 3, 200, 0])
    prob = M.forward(p, X)
    ref = _softmax(b3)
    assert np.allclose(prob, ref[None, :], rtol=1e-13, atol=0)
    loss, g = M.loss_grad(p, X, y)
    assert abs(loss - float(np.mean(-np.log(ref[y])))) < 1e-12
    # with W3 = 0 the hidden layers get no gradient
    assert np.all(g[:O_W3] == 0.0)


def test_hand_wired_network():
    # h1 = relu(x) on the first 64 units, h2 = h1, z_j = c * h2_j for j < 64, z_j = 0 otherwise
    p = np.zeros(M.nparams())
    W1 = np.zeros((NH, NI))
    W1[np.arange(NI), np.arange(NI)] = 1.0
    W2 = np.eye(NH)
    W3 = np.zeros((NO, NH))
    c = 0.7
    W3[np.arange(NI), np.arange(NI)] = c
    p[O_W1:O_B1] = W1.ravel()
    p[O_W2:O_B2] = W2.ravel()
    p[O_W3:O_B3] = W3.ravel()
    X = np.random.default_rng(3).normal(size=(5, NI))
    z = np.zeros((5, NO))
    z[:, :NI] = c * np.maximum(X, 0.0)
    assert np.allclose(M.forward(p, X), _softmax(z), rtol=1e-13, atol=1e-16)
    # an asymmetric W1 block: a transposed product would read the wrong column
    p2 = p.copy()
    W1b = W1.copy()
    W1b[0, :] = 0.0
    W1b[0, 5] = 2.0  # unit 0 sees 2 * x_5
    p2[O_W1:O_B1] = W1b.ravel()
    z2 = z.copy()
    z2[:, 0] = c * np.maximum(2.0 * X[:, 5], 0.0)
    assert np.allclose(M.forward(p2, X), _softmax(z2), rtol=1e-13, atol=1e-16)


def test_gradient_central_differences():
    rng = np.random.default_rng(4)
    p = rng.normal(0, 0.15, M.nparams())
    X = rng.normal(size=(4, NI))
    y = rng.integers(0, NO, 4)
    _, g = M.loss_grad(p, X, y)
    blocks = [(O_W1, O_B1), (O_B1, O_W2), (O_W2, O_B2), (O_B2, O_W3), (O_W3, O_B3), (O_B3, O_B3 + NO)]
    idx = np.concatenate([rng.choice(np.arange(a, b), 40, replace=False) for a, b in blocks])
    h = 1e-5
    worst = 0.0
    scale = np.abs(g).max()
    for i in idx:
        pp = p.copy()
        pp[i] += h
        lp, _ = M.loss_grad(pp, X, y)
        pp[i] -= 2 * h
        lm, _ = M.loss_grad(pp, X, y)
        fd = (lp - lm) / (2 * h)
        worst = max(worst, abs(fd - g[i]) / scale)
    assert worst <= 1e-6


def _perfect_quadtree(L, w0=1.0, h0=1.0):
    """Rectangles of a tree whose every box splits into four equal quarters."""
    rects = []
    for l in range(L + 1):
        k = 2 ** l
        for i in range(4 ** l):
            # any order inside a level gives the same statistics; use row-major quarters
            ix, iy = i % k, i // k
            rects.append([ix * w0 / k, (ix + 1) * w0 / k, iy * h0 / k, (iy + 1) * h0 / k])
    return np.array(rects)


def test_features_of_equal_squares():
    L = 4
    f = M.features(_perfect_quadtree(L), L, 12345, 1e-6)
    for l in range(1, 16):
        blk = f[4 * (l - 1):4 * l]
        if l <= L:
            assert np.allclose(blk, [-l, 0.0, 0.0, 0.0], atol=1e-14)
        else:
            assert np.all(blk == 0.0)
    assert abs(f[60] - math.log10(12345)) < 1e-14
    assert abs(f[61] + 6.0) < 1e-14
    assert f[62] == L / 16 and f[63] == 0.0


def test_features_of_two_to_one_boxes():
    L = 3
    f = M.features(_perfect_quadtree(L, 2.0, 1.0), L, 999, 1e-3)
    for l in range(1, L + 1):
        assert np.allclose(f[4 * (l - 1):4 * l], [-l, 0.0, 1.0, 1.0], atol=1e-14)


def test_features_of_one_elongated_box():
    L = 1
    r = _perfect_quadtree(L)
    r[1] = [0.0, 0.5, 0.0, 0.5 / 8]  # one level-1 box 8:1, long side 1/2
    f = M.features(r, L, 4, 1e-9)
    ls = np.log2(np.array([0.5, 0.5, 0.5, 0.5]) / 1.0)
    la = np.array([3.0, 0.0, 0.0, 0.0])
    assert np.allclose(f[0:4], [ls.mean(), ls.std(), la.mean(), la.max()], atol=1e-14)
    # a degenerate (zero-width) box: the short side is clamped at 2^-30 of the long one
    r[2] = [0.5, 0.5, 0.0, 0.5]
    f = M.features(r, L, 4, 1e-9)
    assert abs(f[3] - 30.0) < 1e-12


@pytest.mark.parametrize("seed", [0, 1])
def test_features_of_real_tree(seed):
    # on a real median-split tree the level means fall by about one octave per level
    from paper_1006_2269_gb300 import workloads as W
    c = W.uniform(4 ** 5 * 3, 900 + seed)
    _, rects, _ = oracle.tree(c.x, c.y, 5)
    f = M.features(rects, 5, c.x.shape[0], 1e-6)
    means = f[0:20:4]
    assert np.all(np.abs(means + np.arange(1, 6)) < 0.35)
    assert np.all(f[2:20:4] < 1.5)  # nearly square boxes on uniform points
