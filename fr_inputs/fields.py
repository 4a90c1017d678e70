"""Analytic initial fields, evaluated at caller-supplied physical coordinates.

Each function takes coordinates ``x`` of shape [ndims, ...] and returns the
conserved state (rho, rho*v, E) stacked on a leading axis of length ndims+2.
The caller decides where the points are (solution points of its own
discretisation); nothing here knows about the FR method.
"""

from __future__ import annotations

import numpy as np


def _xp(x):
    """Array module of x: numpy, or torch for torch tensors (device inputs)."""
    if type(x).__module__.startswith("torch"):
        import torch
        return torch
    return np


def conserved(rho, vel, p, gamma):
    """(rho, v, p) -> (rho, rho v, E) with E = p/(gamma-1) + rho |v|^2 / 2."""
    xp = _xp(rho)
    ke = 0.5 * rho * sum(v * v for v in vel)
    return xp.stack([rho] + [rho * v for v in vel] + [p / (gamma - 1.0) + ke])


def uniform(x, rho, vel, p, gamma):
    shape = np.shape(x[0])
    ones = np.ones(shape)
    return conserved(rho * ones, [v * ones for v in vel], p * ones, gamma)


def isentropic_vortex(x, S=5.0, M=0.4, R=1.5, gamma=1.4, x0=(0.0, 0.0), t=0.0):
    """Isentropic Euler vortex translating with unit speed along +x.

    The paper's vortex (Sec. 5.1) translates along +y; this is the same field
    mirrored so that the free stream is (1, 0).  At time t the exact solution
    is the initial field shifted by (t, 0).
    """
    X = x[0] - x0[0] - t
    Y = x[1] - x0[1]
    f = (1.0 - X * X - Y * Y) / (2.0 * R * R)
    ef = np.exp(f)
    rho = (1.0 - S * S * M * M * (gamma - 1.0) * ef * ef / (8.0 * np.pi ** 2)) ** (1.0 / (gamma - 1.0))
    vx = 1.0 - S * Y * ef / (2.0 * np.pi * R)
    vy = S * X * ef / (2.0 * np.pi * R)
    p = rho ** gamma / (gamma * M * M)
    return conserved(rho, [vx, vy], p, gamma)


def taylor_green(x, M=0.1, gamma=1.4):
    """3D Taylor-Green vortex, V0 = rho0 = 1, isothermal density."""
    X, Y, Z = x[0], x[1], x[2]
    p0 = 1.0 / (gamma * M * M)
    u = np.sin(X) * np.cos(Y) * np.cos(Z)
    v = -np.cos(X) * np.sin(Y) * np.cos(Z)
    w = np.zeros_like(u)
    p = p0 + (np.cos(2 * X) + np.cos(2 * Y)) * (np.cos(2 * Z) + 2.0) / 16.0
    rho = p / p0
    return conserved(rho, [u, v, w], p, gamma)


def _perturbation_terms(rng, nmodes, ndims):
    ks = np.array([k for k in np.ndindex(*(7,) * ndims)]) - 3
    ks = ks[np.any(ks != 0, axis=1)]
    k = ks[rng.integers(len(ks), size=nmodes)]
    a = rng.uniform(-1.0, 1.0, size=nmodes)
    phi = rng.uniform(0.0, 2 * np.pi, size=nmodes)
    return k, a, phi


def perturbed_taylor_green(x, M=0.1, gamma=1.4, amp=0.01, nmodes=8, seed=1312):
    """Taylor-Green field plus amp * sum_m a_m sin(k_m . x + phi_m) on each of
    rho, u, v, w, p (p scaled by rho0 V0^2 = 1); integer k_m in {-3..3}^3.

    x may be a numpy array or a torch tensor (evaluated where it lives)."""
    xp = _xp(x[0])
    X0, X1, X2 = x[0], x[1], x[2]
    rng = np.random.default_rng(seed)
    p0 = 1.0 / (gamma * M * M)
    u = xp.sin(X0) * xp.cos(X1) * xp.cos(X2)
    v = -xp.cos(X0) * xp.sin(X1) * xp.cos(X2)
    w = xp.zeros_like(u)
    p = p0 + (xp.cos(2 * X0) + xp.cos(2 * X1)) * (xp.cos(2 * X2) + 2.0) / 16.0
    rho = p / p0
    prims = [rho, u, v, w, p]
    out = []
    for q in prims:
        k, a, phi = _perturbation_terms(rng, nmodes, 3)
        d = xp.zeros_like(q)
        for m in range(nmodes):
            arg = float(k[m][0]) * X0 + float(k[m][1]) * X1 + float(k[m][2]) * X2 + float(phi[m])
            d += float(a[m]) * xp.sin(arg)
        out.append(q + amp * d)
    return conserved(out[0], out[1:4], out[4], gamma)


def smooth_random(x, gamma=1.4, amp=0.1, nmodes=6, seed=0, rho0=1.0, p0=1.0, vel0=None,
                  period=None):
    """Positive smooth random state for parity tests.

    rho, p = base * (1 + amp*s), v = vel0 + amp*s with s sums of sinusoids.
    ``period`` (scalar) makes every wave number an integer multiple of
    2*pi/period so the field is periodic on such boxes.
    """
    ndims = x.shape[0]
    rng = np.random.default_rng(seed)
    vel0 = np.zeros(ndims) if vel0 is None else np.asarray(vel0, float)
    scale = 1.0 if period is None else 2 * np.pi / period

    def s():
        acc = np.zeros(np.shape(x[0]))
        for _ in range(nmodes):
            k = rng.integers(-3, 4, size=ndims) * scale
            if period is None:
                k = k + rng.uniform(-0.5, 0.5, size=ndims)
            acc += rng.uniform(-1, 1) * np.sin(np.tensordot(k, x, axes=1) + rng.uniform(0, 2 * np.pi))
        return acc / np.sqrt(nmodes)

    rho = rho0 * (1.0 + amp * s())
    vel = [vel0[d] + amp * s() for d in range(ndims)]
    p = p0 * (1.0 + amp * s())
    return conserved(rho, vel, p, gamma)


def couette(x, gamma=1.4, prandtl=0.72, cpTw=1005.0 * 300.0, vw=69.445, p=1e5, h=1.0):
    """Steady compressible Couette flow between isothermal plates at y = 0
    (at rest) and y = h (moving at vw along x), constant viscosity (Sec. 5.2):
    rho = gamma/(gamma-1) 2p / (2 C_pT_w + Pr vw^2 phi (1 - phi)), v = vw phi x,
    p constant, phi = y / h."""
    phi = x[1] / h
    rho = gamma / (gamma - 1.0) * 2.0 * p / (2.0 * cpTw + prandtl * vw ** 2 * phi * (1.0 - phi))
    zero = 0.0 * phi
    return conserved(rho, [vw * phi, zero], p + zero, gamma)


def couette_mean_density(gamma=1.4, prandtl=0.72, cpTw=1005.0 * 300.0, vw=69.445, p=1e5, n=64):
    """<rho(phi)> over phi in [0, 1] (Gauss-Legendre), the constant initial
    density of the Couette runs (Sec. 5.2)."""
    t, w = np.polynomial.legendre.leggauss(n)
    phi = 0.5 * (t + 1.0)
    rho = gamma / (gamma - 1.0) * 2.0 * p / (2.0 * cpTw + prandtl * vw ** 2 * phi * (1.0 - phi))
    return float(0.5 * np.sum(w * rho))
