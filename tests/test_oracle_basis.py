"""Pins of the oracle's 1D reference element (Sec. 2.1, Sec. 3) against
closed forms and exactness properties."""
import numpy as np
import pytest

from oracle import fem


def test_gll_closed_forms():
    assert np.allclose(fem.gll_points(1), [-1, 1], atol=0)
    assert np.allclose(fem.gll_points(2), [-1, 0, 1], atol=1e-16)
    s5 = 1 / np.sqrt(5)
    assert np.allclose(fem.gll_points(3), [-1, -s5, s5, 1], atol=1e-15)
    s37 = np.sqrt(3 / 7)
    assert np.allclose(fem.gll_points(4), [-1, -s37, 0, s37, 1], atol=1e-15)
    a = np.sqrt((7 - 2 * np.sqrt(7)) / 21)
    b = np.sqrt((7 + 2 * np.sqrt(7)) / 21)
    assert np.allclose(fem.gll_points(5), [-1, -b, -a, a, b, 1], atol=1e-15)


@pytest.mark.parametrize("k", range(1, 9))
def test_gll_quadrature_exactness(k):
    # The GLL rule with weights 2 / (k (k+1) P_k(x_i)^2) is exact up to
    # degree 2k-1; this only holds if the nodes are the GLL points.
    x = fem.gll_points(k)
    Pk = np.polynomial.legendre.Legendre.basis(k)(x)
    w = 2.0 / (k * (k + 1) * Pk ** 2)
    for m in range(2 * k):
        exact = 0.0 if m % 2 else 2.0 / (m + 1)
        assert abs(w @ x ** m - exact) < 1e-14


@pytest.mark.parametrize("n", range(1, 10))
def test_gauss_exactness(n):
    x, w = fem.gauss_rule(n)
    for m in range(2 * n):
        exact = 0.0 if m % 2 else 2.0 / (m + 1)
        assert abs(w @ x ** m - exact) < 1e-14


@pytest.mark.parametrize("k", range(1, 9))
def test_lagrange_cardinal_and_derivative(k):
    nodes = fem.gll_points(k)
    assert np.allclose(fem.lagrange_values(nodes, nodes), np.eye(k + 1),
                       atol=1e-14)
    x = np.linspace(-1, 1, 7)
    D = fem.lagrange_derivatives(nodes, x)
    V = fem.lagrange_values(nodes, x)
    for m in range(k + 1):
        assert np.allclose(V @ nodes ** m, x ** m, atol=1e-12)
        ref = m * x ** (m - 1) if m else np.zeros_like(x)
        assert np.allclose(D @ nodes ** m, ref, atol=1e-11)


def test_basis3d_partition_of_unity():
    pts = np.random.default_rng(0).uniform(-1, 1, (11, 3))
    val, grad = fem.basis3d(3, pts)
    assert np.allclose(val.sum(1), 1.0, atol=1e-13)
    assert np.allclose(grad.sum(1), 0.0, atol=1e-12)
