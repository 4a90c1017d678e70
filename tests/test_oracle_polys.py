"""Pins for oracle.polys against library routines and closed forms."""
import numpy as np
import numpy.polynomial.legendre as npleg
from scipy.special import eval_jacobi

from oracle.polys import gauss_legendre, legendre, jacobi, lagrange


def test_gauss_legendre_matches_numpy_leggauss():
    for n in range(1, 12):
        x, w = gauss_legendre(n)
        xr, wr = npleg.leggauss(n)
        assert np.allclose(x, xr, atol=1e-14, rtol=0)
        assert np.allclose(w, wr, atol=1e-14, rtol=0)


def test_gauss_legendre_closed_form_two_points():
    x, w = gauss_legendre(2)
    assert np.allclose(x, [-1 / np.sqrt(3), 1 / np.sqrt(3)], atol=1e-15)
    assert np.allclose(w, [1.0, 1.0], atol=1e-15)


def test_gauss_legendre_exactness():
    for n in range(1, 8):
        x, w = gauss_legendre(n)
        for k in range(2 * n):
            exact = 0.0 if k % 2 else 2.0 / (k + 1)
            assert abs(np.dot(w, x ** k) - exact) < 1e-14


def test_legendre_values_and_derivatives():
    x = np.linspace(-1, 1, 17)
    for n in range(0, 9):
        c = np.zeros(n + 1); c[n] = 1.0
        p, d = legendre(n, x)
        assert np.allclose(p, npleg.legval(x, c), atol=1e-13)
        assert np.allclose(d, npleg.legval(x, npleg.legder(c)), atol=1e-12)


def test_jacobi_matches_scipy():
    x = np.linspace(-0.95, 0.95, 13)
    for n in range(0, 7):
        for a in (0.0, 1.0, 3.0, 5.0):
            p, d = jacobi(n, a, 0.0, x)
            assert np.allclose(p, eval_jacobi(n, a, 0.0, x), atol=1e-12)
            h = 1e-6
            fd = (eval_jacobi(n, a, 0.0, x + h) - eval_jacobi(n, a, 0.0, x - h)) / (2 * h)
            assert np.allclose(d, fd, atol=1e-6 * max(1.0, np.abs(fd).max()))


def test_lagrange_kronecker_and_derivative():
    nodes = np.array([-0.9, -0.2, 0.4, 1.0])
    L, dL = lagrange(nodes, nodes)
    assert np.allclose(L, np.eye(4), atol=1e-15)
    x = np.linspace(-1, 1, 9)
    L, dL = lagrange(nodes, x)
    for j in range(4):
        y = np.zeros(4); y[j] = 1.0
        c = np.polyfit(nodes, y, 3)
        assert np.allclose(L[j], np.polyval(c, x), atol=1e-12)
        assert np.allclose(dL[j], np.polyval(np.polyder(c), x), atol=1e-11)
