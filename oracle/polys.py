"""One-dimensional polynomials and quadrature for the oracle (FP64).

* Gauss-Legendre points/weights by the Golub-Welsch eigenvalue method.
* Legendre and Jacobi polynomials (and derivatives) by their three-term
  recurrences.
* Lagrange interpolation through arbitrary nodes.

These are the building blocks of the spanning basis psi and the point sets of
Sec. 2 (solution/flux points) and of the quadrature used in the L2 error
functional of Sec. 5.
"""

from __future__ import annotations

import numpy as np


def gauss_legendre(n: int):
    """n-point Gauss-Legendre rule on [-1, 1] (Golub-Welsch)."""
    if n == 1:
        return np.array([0.0]), np.array([2.0])
    k = np.arange(1, n)
    off = k / np.sqrt(4.0 * k * k - 1.0)
    T = np.diag(off, 1) + np.diag(off, -1)
    x, V = np.linalg.eigh(T)
    w = 2.0 * V[0, :] ** 2
    # symmetrise against round-off
    x = 0.5 * (x - x[::-1])
    w = 0.5 * (w + w[::-1])
    return x, w


def legendre(n: int, x):
    """P_n(x) and P_n'(x) by the Bonnet recurrence."""
    x = np.asarray(x, dtype=np.result_type(x, np.float64))
    p0, p1 = np.ones_like(x), x
    d0, d1 = np.zeros_like(x), np.ones_like(x)
    if n == 0:
        return p0, d0
    for k in range(1, n):
        p2 = ((2 * k + 1) * x * p1 - k * p0) / (k + 1)
        d2 = d0 + (2 * k + 1) * p1          # P'_{k+1} = P'_{k-1} + (2k+1) P_k
        p0, p1, d0, d1 = p1, p2, d1, d2
    return p1, d1


def jacobi(n: int, a: float, b: float, x):
    """Jacobi P_n^{(a,b)}(x) and its derivative."""
    x = np.asarray(x, dtype=np.float64)
    if n == 0:
        return np.ones_like(x), np.zeros_like(x)
    p0 = np.ones_like(x)
    p1 = 0.5 * (a - b + (a + b + 2.0) * x)
    for k in range(2, n + 1):
        c = 2.0 * k + a + b
        a1 = 2.0 * k * (k + a + b) * (c - 2.0)
        a2 = (c - 1.0) * (a * a - b * b)
        a3 = (c - 2.0) * (c - 1.0) * c
        a4 = 2.0 * (k + a - 1.0) * (k + b - 1.0) * c
        p0, p1 = p1, ((a2 + a3 * x) * p1 - a4 * p0) / a1
    pn = p1
    # d/dx P_n^{(a,b)} = (n+a+b+1)/2 P_{n-1}^{(a+1,b+1)}
    dn = 0.5 * (n + a + b + 1.0) * jacobi(n - 1, a + 1.0, b + 1.0, x)[0]
    return pn, dn


def lagrange(nodes, x):
    """Values and derivatives of the Lagrange polynomials through ``nodes``.

    Returns L[j, ...] = l_j(x) and dL[j, ...] = l_j'(x).
    """
    nodes = np.asarray(nodes, np.float64)
    x = np.asarray(x, np.float64)
    n = len(nodes)
    L = np.ones((n,) + x.shape)
    dL = np.zeros((n,) + x.shape)
    for j in range(n):
        for m in range(n):
            if m == j:
                continue
            den = nodes[j] - nodes[m]
            # product rule: d(L*(x-xm)/den) = dL*(x-xm)/den + L/den
            dL[j] = dL[j] * (x - nodes[m]) / den + L[j] / den
            L[j] = L[j] * (x - nodes[m]) / den
    return L, dL
