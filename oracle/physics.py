"""Governing systems: Euler and compressible Navier-Stokes (Sec. 4), the
Rusanov Riemann solver (App. B), LDG common values (Sec. 4.3) and boundary
ghost states (App. C).

Array conventions: a state u has the variable index first, u[alpha, ...] with
alpha = (rho, rho v_x, rho v_y[, rho v_z], E).  Gradients and fluxes have the
direction first: q[j, alpha, ...] = d u_alpha / d x_j and f[i, alpha, ...] is
the i-th spatial component of the flux of variable alpha.

Every routine is written so that it also works on complex arrays (the oracle's
complex-step derivative): |.| is replaced by sign(Re z) z.
"""

from __future__ import annotations

import numpy as np


def cabs(z):
    """|z| for real z; sign(Re z) * z for complex z (complex-step friendly)."""
    if np.iscomplexobj(z):
        return np.where(z.real >= 0.0, z, -z)
    return np.abs(z)


def primitives(u, gamma):
    """rho, velocity list, pressure from conserved u (Eq. idealgas)."""
    nd = u.shape[0] - 2
    rho = u[0]
    v = [u[1 + i] / rho for i in range(nd)]
    E = u[nd + 1]
    p = (gamma - 1.0) * (E - 0.5 * rho * sum(vi * vi for vi in v))
    return rho, v, p


def inviscid_flux(u, gamma):
    """f^(inv) of Eq. eulerflux: returns f[i, alpha, ...]."""
    nd = u.shape[0] - 2
    rho, v, p = primitives(u, gamma)
    E = u[nd + 1]
    f = np.empty((nd,) + u.shape, dtype=u.dtype)
    for i in range(nd):
        f[i, 0] = rho * v[i]
        for j in range(nd):
            f[i, 1 + j] = rho * v[j] * v[i] + (p if i == j else 0.0)
        f[i, nd + 1] = v[i] * (E + p)
    return f


def viscous_flux(u, q, gamma, mu, prandtl):
    """f^(vis) of Eq. visflux for constant mu.

    Delta dT = (mu C_p / Pr) dT with T = p / (rho C_v (gamma-1)) gives
    Delta dT = mu gamma / (Pr (gamma-1)) d(p/rho); C_p cancels.  Velocity and
    p/rho gradients follow from the conserved gradients by the quotient rule.
    """
    nd = u.shape[0] - 2
    rho, v, p = primitives(u, gamma)
    drho = q[:, 0]
    dm = [q[:, 1 + i] for i in range(nd)]        # dm[i][j] = d(rho v_i)/dx_j
    dE = q[:, nd + 1]
    # dv[i][j] = d v_i / d x_j
    dv = [[(dm[i][j] - v[i] * drho[j]) / rho for j in range(nd)] for i in range(nd)]
    # dp = (gamma-1)(dE - v.dm + |v|^2 drho / 2)
    v2 = sum(vi * vi for vi in v)
    dp = [(gamma - 1.0) * (dE[j] - sum(v[i] * dm[i][j] for i in range(nd)) + 0.5 * v2 * drho[j])
          for j in range(nd)]
    # d(p/rho) = (dp rho - p drho) / rho^2
    dpr = [(dp[j] * rho - p * drho[j]) / (rho * rho) for j in range(nd)]
    div = sum(dv[i][i] for i in range(nd))
    T = [[mu * (dv[j][i] + dv[i][j]) - (2.0 / 3.0 * mu * div if i == j else 0.0)
          for j in range(nd)] for i in range(nd)]   # T[i][j] = mu(d_i v_j + d_j v_i) - ...
    kappa = mu * gamma / (prandtl * (gamma - 1.0))
    f = np.zeros((nd,) + u.shape, dtype=np.result_type(u, q))
    for i in range(nd):
        for j in range(nd):
            f[i, 1 + j] = T[i][j]
        f[i, nd + 1] = sum(v[j] * T[j][i] for j in range(nd)) + kappa * dpr[i]
    return f


def rusanov(uL, uR, n, gamma):
    """Rusanov (local Lax-Friedrichs) common inviscid normal flux, App. B.

    n[i, ...] is the unit normal of the L side.
    """
    nd = uL.shape[0] - 2
    fL = inviscid_flux(uL, gamma)
    fR = inviscid_flux(uR, gamma)
    rhoL, vL, pL = primitives(uL, gamma)
    rhoR, vR, pR = primitives(uR, gamma)
    nv = sum(n[i] * (vL[i] + vR[i]) for i in range(nd))
    s = np.sqrt(gamma * (pL + pR) / (rhoL + rhoR)) + 0.5 * cabs(nv)
    nf = sum(n[i] * (fL[i] + fR[i]) for i in range(nd))
    return 0.5 * nf + 0.5 * s * (uL - uR)


def ldg_common_solution(uL, uR, beta):
    """C(u_L, u_R) = (1/2 - beta) u_L + (1/2 + beta) u_R (Sec. 4.3)."""
    return (0.5 - beta) * uL + (0.5 + beta) * uR


def ldg_viscous_normal(fvL, fvR, n, beta):
    """n_L . {(1/2 + beta) f_vis,L + (1/2 - beta) f_vis,R} (Sec. 4.3)."""
    nd = fvL.shape[0]
    return sum(n[i] * ((0.5 + beta) * fvL[i] + (0.5 - beta) * fvR[i]) for i in range(nd))


# ---------------------------------------------------------------- boundaries
BC_INFLOW, BC_OUTFLOW, BC_WALL, BC_WALL2 = 0, 1, 2, 3


def ghost_states(btype, uL, qL, prm):
    """Ghost solutions for the inviscid and LDG parts and the ghost gradient
    (App. C).  Returns (u_inv, u_ldg, q_ghost)."""
    gamma = prm["gamma"]
    nd = uL.shape[0] - 2
    shape = uL.shape[1:]
    if btype == BC_INFLOW:
        rho = prm["bc_rho"]
        v = prm["bc_v"][:nd]
        p = prm["bc_p"]
        g = np.empty_like(uL)
        g[0] = rho
        for i in range(nd):
            g[1 + i] = rho * v[i]
        g[nd + 1] = p / (gamma - 1.0) + 0.5 * rho * sum(vi * vi for vi in v)
        qg = None if qL is None else np.zeros_like(qL)
        return g, g, qg
    if btype == BC_OUTFLOW:
        rho, v, _ = primitives(uL, gamma)
        g = np.empty_like(uL)
        g[0] = rho
        for i in range(nd):
            g[1 + i] = uL[1 + i]
        g[nd + 1] = prm["outflow_p"] / (gamma - 1.0) + 0.5 * rho * sum(vi * vi for vi in v)
        qg = None if qL is None else np.zeros_like(qL)
        return g, g, qg
    if btype in (BC_WALL, BC_WALL2):
        # BC_WALL2: a second isothermal wall (same C_p T_w) moving at wall2_v,
        # e.g. the moving plate of Couette flow (Sec. 5.2)
        rho, v, _ = primitives(uL, gamma)
        vw = prm["wall_v" if btype == BC_WALL else "wall2_v"][:nd]
        cpTw = prm["wall_cpTw"]
        gi = np.empty_like(uL)
        vm = [2.0 * vw[i] - v[i] for i in range(nd)]
        gi[0] = rho
        for i in range(nd):
            gi[1 + i] = rho * vm[i]
        gi[nd + 1] = rho * (cpTw / gamma + 0.5 * sum(x * x for x in vm))
        gl = np.empty_like(uL)
        gl[0] = rho
        for i in range(nd):
            gl[1 + i] = rho * vw[i]
        gl[nd + 1] = rho * (cpTw / gamma + 0.5 * sum(x * x for x in vw))
        return gi, gl, qL
    raise ValueError(f"unknown boundary type {btype}")
