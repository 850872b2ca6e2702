"""Pins of the oracle's 1D basis (Sec. Spatial discretization) to textbook values."""
import numpy as np
import pytest

from oracle import basis


def test_gll_textbook_tables():
    # p = 2: Simpson's rule; p = 4: the 5-point Lobatto rule (nodes 0, +-sqrt(3/7), +-1).
    x, w = basis.gll_points(2)
    assert np.allclose(x, [-1, 0, 1], atol=1e-15)
    assert np.allclose(w, [1 / 3, 4 / 3, 1 / 3], atol=1e-15)
    x, w = basis.gll_points(4)
    r = np.sqrt(3.0 / 7.0)
    assert np.allclose(x, [-1, -r, 0, r, 1], atol=1e-15)
    assert np.allclose(w, [1 / 10, 49 / 90, 32 / 45, 49 / 90, 1 / 10], atol=1e-15)


@pytest.mark.parametrize("p", range(1, 9))
def test_gll_exactness(p):
    x, w = basis.gll_points(p)
    assert abs(w.sum() - 2.0) < 1e-14
    for k in range(0, 2 * p):             # exact through degree 2p-1
        exact = 2.0 / (k + 1) if k % 2 == 0 else 0.0
        assert abs((w * x ** k).sum() - exact) < 1e-13
    k = 2 * p                              # not exact at degree 2p
    assert abs((w * x ** k).sum() - 2.0 / (k + 1)) > 1e-6


@pytest.mark.parametrize("n", range(1, 8))
def test_gauss_exactness(n):
    x, w = basis.gauss_points(n)
    for k in range(0, 2 * n):
        exact = 2.0 / (k + 1) if k % 2 == 0 else 0.0
        assert abs((w * x ** k).sum() - exact) < 1e-13


@pytest.mark.parametrize("p", [1, 2, 3, 4, 5])
def test_lagrange_properties(p):
    nodes, _ = basis.gll_points(p)
    L = basis.lagrange(nodes, nodes)
    assert np.array_equal(L, np.eye(p + 1))           # Kronecker delta, exactly
    xi = np.linspace(-1, 1, 37)
    assert np.allclose(basis.lagrange(nodes, xi).sum(axis=1), 1.0, atol=1e-13)
    d = basis.lagrange_deriv(nodes, xi)
    assert np.allclose(d.sum(axis=1), 0.0, atol=1e-11)
    eps = 1e-6
    fd = (basis.lagrange(nodes, xi + eps) - basis.lagrange(nodes, xi - eps)) / (2 * eps)
    assert np.allclose(d, fd, atol=1e-7)
    # Interpolation of a degree-p polynomial is exact.
    f = lambda t: 0.3 * t ** p - 0.7 * t + 0.2
    assert np.allclose(basis.lagrange(nodes, xi) @ f(nodes), f(xi), atol=1e-13)
