"""Explicit time steppers of the FR system besides RK4 (test infrastructure).

The paper lists forward Euler, classical RK4 and DOPRI5 among the time
steppers of its implementation (Sec. 3, table of functionality) without
further detail.  This module writes them out for a right-hand side given as
a callable on lists of per-block arrays:

* forward Euler: u_{n+1} = u_n + dt R(u_n);
* DOPRI5: the seven-stage embedded pair of Dormand and Prince (1980), with
  the 5th-order solution propagated and the 4th-order one used only for the
  error estimate E = u5 - u4 = dt sum_j (b_j - bs_j) k_j.  The last stage is
  evaluated at the new solution (row 7 of A equals b), so its slope is the
  first slope of the next step ("first same as last").
* error norm (Hairer, Norsett and Wanner, Sec. II.4):
  ||E|| = sqrt(mean_i (E_i / (atol + rtol max(|u_n,i|, |u_n+1,i|)))^2).

The tableau is the published one, as exact fractions.
"""

from __future__ import annotations

from fractions import Fraction as Fr

import numpy as np

# Dormand-Prince 5(4): nodes c, matrix A (strictly lower), weights b (order 5), bs (order 4)
DP_C = [Fr(0), Fr(1, 5), Fr(3, 10), Fr(4, 5), Fr(8, 9), Fr(1), Fr(1)]
DP_A = [
    [],
    [Fr(1, 5)],
    [Fr(3, 40), Fr(9, 40)],
    [Fr(44, 45), Fr(-56, 15), Fr(32, 9)],
    [Fr(19372, 6561), Fr(-25360, 2187), Fr(64448, 6561), Fr(-212, 729)],
    [Fr(9017, 3168), Fr(-355, 33), Fr(46732, 5247), Fr(49, 176), Fr(-5103, 18656)],
    [Fr(35, 384), Fr(0), Fr(500, 1113), Fr(125, 192), Fr(-2187, 6784), Fr(11, 84)],
]
DP_B = [Fr(35, 384), Fr(0), Fr(500, 1113), Fr(125, 192), Fr(-2187, 6784), Fr(11, 84), Fr(0)]
DP_BS = [Fr(5179, 57600), Fr(0), Fr(7571, 16695), Fr(393, 640), Fr(-92097, 339200), Fr(187, 2100), Fr(1, 40)]


def euler(rhs, U, dt, nsteps=1):
    """Forward Euler."""
    U = [u.copy() for u in U]
    for _ in range(nsteps):
        K = rhs(U)
        U = [u + dt * k for u, k in zip(U, K)]
    return U


def dopri5_step(rhs, U, dt, k1=None):
    """One DOPRI5 step: returns (U_{n+1} (order 5), E = U5 - U4, slope at U_{n+1})."""
    ks = [rhs(U) if k1 is None else k1]
    for i in range(1, 7):
        Y = [u + dt * sum(float(a) * k[b] for a, k in zip(DP_A[i], ks)) for b, u in enumerate(U)]
        ks.append(rhs(Y))
    # row 7 of A is b: the last stage input Y is the 5th-order solution
    U5 = Y
    E = [dt * sum(float(bb - bs) * k[b] for bb, bs, k in zip(DP_B, DP_BS, ks)) for b in range(len(U))]
    return U5, E, ks[-1]


def error_norm(U0, U1, E, atol, rtol):
    """RMS of E scaled by atol + rtol max(|U0|, |U1|) over every entry of every block."""
    s, n = 0.0, 0
    for u0, u1, e in zip(U0, U1, E):
        sc = atol + rtol * np.maximum(np.abs(u0), np.abs(u1))
        s += float(np.sum(np.abs(e / sc) ** 2))
        n += e.size
    return np.sqrt(s / n)


def dopri5(rhs, U, dt, nsteps=1, atol=1e-6, rtol=1e-6):
    """nsteps fixed DOPRI5 steps (slope reuse between steps); returns
    (U_N, error norm of the last step)."""
    k1 = None
    err = 0.0
    for _ in range(nsteps):
        U1, E, k1 = dopri5_step(rhs, U, dt, k1)
        err = error_norm(U, U1, E, atol, rtol)
        U = U1
    return U, err
