"""Pins for oracle.lagrange against closed forms (Sec. 3.2: q-th order
Lagrange interpolation on (q+1) nodes per axis)."""
import numpy as np
import pytest

from oracle import lagrange


@pytest.mark.parametrize("p", [1, 2, 3, 4, 5, 6])
def test_reproduces_polynomials(p):
    t = np.linspace(-0.7, p + 0.7, 41)
    w = lagrange.weights(t, p)
    nodes = np.arange(p + 1)
    for deg in range(p + 1):
        assert np.allclose(w @ nodes.astype(float) ** deg, t ** deg, rtol=0, atol=1e-11 * (p + 1) ** deg)
    # degree p+1 is NOT reproduced: the error is the nodal polynomial
    err = w @ nodes.astype(float) ** (p + 1) - t ** (p + 1)
    nodal = np.prod([t - j for j in nodes], axis=0)
    assert np.allclose(err, -nodal, atol=1e-9)


@pytest.mark.parametrize("p", [1, 2, 4, 5])
def test_derivative_weights(p):
    t = np.linspace(0.1, p - 0.1, 17)
    dw = lagrange.dweights(t, p)
    nodes = np.arange(p + 1).astype(float)
    for deg in range(1, p + 1):
        assert np.allclose(dw @ nodes ** deg, deg * t ** (deg - 1), atol=1e-10 * (p + 1) ** deg)
    assert np.allclose(dw.sum(axis=1), 0.0, atol=1e-12)
    # against a central difference of the weights themselves
    e = 1e-6
    fd = (lagrange.weights(t + e, p) - lagrange.weights(t - e, p)) / (2 * e)
    assert np.allclose(dw, fd, atol=1e-7)


def test_stencil_rule_even_odd_and_clamp():
    h, n = 0.1, 11
    x = np.array([0.0, 0.04, 0.26, 0.5, 0.74, 0.96, 1.0])
    s4, t4 = lagrange.stencil_start(x, h, n, 4)
    # even p: nearest node minus p/2, clamped into [0, n-1-p]
    assert list(s4) == [0, 0, 1, 3, 5, 6, 6]
    assert np.allclose(t4, x / h - s4)
    s3, t3 = lagrange.stencil_start(x, h, n, 3)
    # odd p: cell index minus (p-1)/2, clamped into [0, n-1-p]
    assert list(s3) == [0, 0, 1, 4, 6, 7, 7]
    # every point of the closed interval [0, (n-1)h] lies inside its stencil
    xx = np.linspace(0, (n - 1) * h, 1001)
    for p in (2, 3, 4, 5):
        s, t = lagrange.stencil_start(xx, h, n, p)
        assert np.all(t >= -1e-12) and np.all(t <= p + 1e-12)
    # shifted grid (far observer grid)
    s, t = lagrange.stencil_start(np.array([0.55]), 0.1, 10, 4, shift=0.05)
    assert s[0] == 3 and abs(t[0] - 2.0) < 1e-12


def test_box_index():
    b = lagrange.box_index(np.array([0.0, 0.099, 0.1, 0.95, 1.0]), 0.1, 10)
    assert list(b) == [0, 0, 1, 9, 9]


@pytest.mark.parametrize("p", [2, 3, 4])
def test_points_of_a_box_share_one_stencil(p):
    h, n = 0.1, 12
    x = np.random.default_rng(0).random(4000) * (n - 1) * h
    x = np.concatenate([x, [0.0, (n - 1) * h, 0.05, 0.15, 1.05]])
    B = lagrange.stencil_box(x, h, n, p)
    s, _ = lagrange.stencil_start(x, h, n, p)
    lo = p // 2 if p % 2 == 0 else (p - 1) // 2
    assert np.array_equal(s, np.clip(B - lo, 0, n - 1 - p))
    assert B.min() >= 0 and B.max() <= (n - 1 if p % 2 == 0 else n - 2)
