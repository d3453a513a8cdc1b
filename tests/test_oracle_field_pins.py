"""Pins of the oracle's complex field F_i = sum_{j != i} -q_j / (z_i - z_j), the kernel of the
paper's first experiment (Section 5), on the CPU.

Closed forms: two points; the n-th roots of unity, where sum_{j != i} 1/(z_i - z_j) =
(n - 1) / (2 z_i) (from P''/(2P') of z^n - 1).  The field is the gradient of the potential of
Eq. (1.1) (Re F = -dphi/dx, Im F = +dphi/dy), checked by central differences of the direct
potential.  The method's field: equal to the direct field when there is no far field (one level
of boxes or none), and converging geometrically in p like theta^(p+1).
"""
import math

import numpy as np
import pytest

import oracle
from paper_1006_2269_gb300 import workloads as W


def test_two_points():
    x = np.array([0.3, -1.1])
    y = np.array([0.7, 0.2])
    q = np.array([2.0, -0.5])
    f = oracle.direct_field(x, y, q)
    z = x + 1j * y
    assert abs(f[0] - (-q[1] / (z[0] - z[1]))) < 1e-15
    assert abs(f[1] - (-q[0] / (z[1] - z[0]))) < 1e-15


@pytest.mark.parametrize("n", [3, 8, 101])
def test_roots_of_unity(n):
    t = 2 * np.pi * np.arange(n) / n
    z = np.exp(1j * t)
    f = oracle.direct_field(z.real, z.imag, np.ones(n))
    assert np.max(np.abs(f - (-(n - 1) / (2 * z)))) < 1e-12 * n


def test_field_is_gradient_of_potential():
    c = W.uniform(200, 31)
    h = 1e-6
    for i in (0, 17, 123):
        xp, xm = c.x.copy(), c.x.copy()
        xp[i] += h
        xm[i] -= h
        dphidx = (oracle.direct(xp, c.y, c.q, [i])[0] - oracle.direct(xm, c.y, c.q, [i])[0]) / (2 * h)
        yp, ym = c.y.copy(), c.y.copy()
        yp[i] += h
        ym[i] -= h
        dphidy = (oracle.direct(c.x, yp, c.q, [i])[0] - oracle.direct(c.x, ym, c.q, [i])[0]) / (2 * h)
        f = oracle.direct_field(c.x, c.y, c.q, [i])[0]
        scale = abs(f) + 1.0
        assert abs(f.real + dphidx) < 1e-6 * scale
        assert abs(f.imag - dphidy) < 1e-6 * scale


@pytest.mark.parametrize("L", [0, 1])
def test_method_without_far_field_is_direct(L):
    # with L = 0 every pair is near; with L = 1 no pair of the four boxes is weak
    c = W.normal(700, 32)
    f = oracle.fmm_field(c.x, c.y, c.q, L, 10, 0.5)
    d = oracle.direct_field(c.x, c.y, c.q)
    assert np.max(np.abs(f - d)) <= 1e-13 * np.max(np.abs(d))


def test_method_converges_like_theta_power():
    c = W.disc_uniform(6000, 33)
    d = oracle.direct_field(c.x, c.y, c.q)
    errs = []
    for p in (4, 8, 12, 16):
        f = oracle.fmm_field(c.x, c.y, c.q, 4, p, 0.5)
        errs.append(np.max(np.abs(f - d)) / np.max(np.abs(d)))
    errs = np.array(errs)
    # every four more orders cut the error at least 8-fold (theta^4 = 1/16, with a margin of 2)
    assert np.all(errs[1:] <= errs[:-1] / 8)
    # and the level is that of the Section 3 estimate theta^(p+1) / (1 - theta)^2
    assert np.all(errs <= 0.5 ** (np.array([4, 8, 12, 16]) + 1) / 0.25)
