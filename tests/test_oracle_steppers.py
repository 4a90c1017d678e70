"""Pins of the oracle's forward Euler and DOPRI5 steppers (Sec. 3 lists both
beside RK4): Butcher's order conditions on the tableau, the stability
polynomials on the linear test equation, and observed convergence orders."""

from fractions import Fraction as Fr

import numpy as np
import pytest

from oracle import steppers as S


# ----------------------------------------------------------- rooted trees
def _trees(order):
    """All rooted trees with `order` vertices, as sorted tuples of subtrees."""
    if order == 1:
        return [()]
    out = set()

    def parts(n, maxpart):                      # partitions of n into parts <= maxpart, non-increasing
        if n == 0:
            yield []
            return
        for k in range(min(n, maxpart), 0, -1):
            for rest in parts(n - k, k):
                yield [k] + rest

    for p in parts(order - 1, order - 1):
        def combos(idx):
            if idx == len(p):
                yield []
                return
            for t in _trees(p[idx]):
                for rest in combos(idx + 1):
                    yield [t] + rest
        for c in combos(0):
            out.add(tuple(sorted(c)))
    return sorted(out)


def _size(t):
    return 1 + sum(_size(c) for c in t)


def _density(t):
    g = _size(t)
    for c in t:
        g *= _density(c)
    return g


def _phi(t, A):
    """Vector of internal elementary weights of tree t."""
    s = len(A)
    v = [Fr(1)] * s
    for c in t:
        w = _phi(c, A)
        aw = [sum((A[i][j] if j < len(A[i]) else Fr(0)) * w[j] for j in range(s)) for i in range(s)]
        v = [v[i] * aw[i] for i in range(s)]
    return v


def _satisfies(b, A, t):
    return sum(bi * pi for bi, pi in zip(b, _phi(t, A))) == Fr(1, _density(t))


def test_tree_counts():
    # number of rooted trees with n vertices: 1, 1, 2, 4, 9, 20 (OEIS A000081)
    assert [len(_trees(n)) for n in range(1, 7)] == [1, 1, 2, 4, 9, 20]


def test_dopri5_order_conditions():
    A, b, bs, c = S.DP_A, S.DP_B, S.DP_BS, S.DP_C
    for i in range(7):
        assert sum(A[i]) == c[i]                      # row-sum condition
    for n in range(1, 6):
        for t in _trees(n):
            assert _satisfies(b, A, t), ("b", n, t)
    assert not all(_satisfies(b, A, t) for t in _trees(6))    # exactly order 5
    for n in range(1, 5):
        for t in _trees(n):
            assert _satisfies(bs, A, t), ("bs", n, t)
    assert not all(_satisfies(bs, A, t) for t in _trees(5))   # exactly order 4
    assert A[6] + [Fr(0)] == b                        # last stage at the new solution


# ----------------------------------------------------------- linear test equation
def _linear(lam):
    return lambda U: [lam * u for u in U]


@pytest.mark.parametrize("z", [0.1, 0.5, 1.3, -2.0 + 1.0j])
def test_stability_polynomials(z):
    lam = -0.7 + 0.4j
    U = [np.ones((3, 2, 4), complex)]
    dt = z / lam
    e = S.euler(_linear(lam), U, dt, 1)[0]
    assert np.allclose(e, 1 + z, rtol=1e-14)
    u5, _ = S.dopri5(_linear(lam), U, dt, 1)
    expect = sum(z ** k / np.prod(range(1, k + 1)) for k in range(6)) + z ** 6 / 600
    assert np.allclose(u5[0], expect, rtol=1e-13)


def test_fsal_reuse_equals_separate_steps():
    f = lambda U: [-u * u + np.sin(u) for u in U]
    U = [np.linspace(0.1, 1.0, 12).reshape(3, 2, 2)]
    two, _ = S.dopri5(f, U, 0.05, 2)
    one, _ = S.dopri5(f, U, 0.05, 1)
    one, _ = S.dopri5(f, one, 0.05, 1)
    assert np.array_equal(two[0], one[0])


# ----------------------------------------------------------- a nonlinear ODE with known solution
def _riccati():
    # u' = -u^2, u(0) = u0  =>  u(t) = u0 / (1 + u0 t)
    u0 = np.array([0.5, 1.0, 2.0]).reshape(3, 1, 1)
    return (lambda U: [-u * u for u in U]), [u0], (lambda t: u0 / (1 + u0 * t))


@pytest.mark.parametrize("method,order", [("euler", 1), ("dopri5", 5)])
def test_global_convergence_order(method, order):
    f, U, exact = _riccati()
    T, errs = 1.0, []
    for n in ((8, 16, 32) if method == "euler" else (32, 64, 128)):
        dt = T / n
        if method == "euler":
            u = S.euler(f, U, dt, n)
        else:
            u, _ = S.dopri5(f, U, dt, n)
        errs.append(np.abs(u[0] - exact(T)).max())
    rates = np.log2(np.array(errs[:-1]) / np.array(errs[1:]))
    # DOPRI5's small leading error constant leaves the 6th-order term visible
    # at these steps: the rate falls towards 5 from above
    assert np.all(rates > order - 0.3) and rates[-1] < order + 1.0, rates


def test_error_estimate_is_fifth_order_local_error():
    f, U, _ = _riccati()
    norms = []
    for dt in (0.2, 0.1, 0.05):
        _, E, _ = S.dopri5_step(f, U, dt)
        norms.append(np.abs(E[0]).max())
    rates = np.log2(np.array(norms[:-1]) / np.array(norms[1:]))
    assert np.all(np.abs(rates - 5) < 0.5), rates      # E = u5 - u4 = O(dt^5)


def test_error_norm_definition():
    U0 = [np.array([1.0, -2.0])]
    U1 = [np.array([3.0, 1.0])]
    E = [np.array([0.5, 0.25])]
    # scales: atol + rtol max(|u0|, |u1|) = 0.1 + 0.1 * (3, 2)
    expect = np.sqrt(((0.5 / 0.4) ** 2 + (0.25 / 0.3) ** 2) / 2)
    assert S.error_norm(U0, U1, E, 0.1, 0.1) == pytest.approx(expect, rel=1e-15)
