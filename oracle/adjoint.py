"""Discrete adjoint of the Euler right-hand side and of classical RK4 (FP64).

Not in the paper: the transpose (dR/dU)^T lambda of the FR operator of
Sec. 2 / App. A for the Euler equations, assembled by running the RHS steps
backwards:

    R = -J^-1 [M3 D~ + (M1 - M3 M2) F~],   F~ = adj(J) f(U),
    D~_L = |n|_L F(uL, uR, n),  D~_R = -|n|_R F(uL, uR, n),   uf = M0 U

    mu   = -J^-1 lambda
    g_D  = M3^T mu,  g_F = (M1 - M3 M2)^T mu  (= M1^T mu - M2^T g_D)
    per pair:  a = |n|_L g_D,L - |n|_R g_D,R;  a_uL = (dF/duL)^T a,  a_uR = (dF/duR)^T a
    boundary:  a_ub = (d F(ub, ghost(ub)) / dub)^T (|n| g_D)
    out  = M0^T a_uf + (d f / dU)^T (adj(J)^T g_F)   (point-wise)

The local Jacobians (flux, Rusanov with its ghost states) are taken exactly
by the complex-step method on the oracle's own complex-safe physics.

RK4 adjoint (u_{n+1} = u_n + dt/6 (k1 + 2 k2 + 2 k3 + k4), k_i = R(y_i)):
    w4 = J4^T (dt/6 l);  nu3 = dt/3 l + dt w4;    w3 = J3^T nu3
    nu2 = dt/3 l + dt/2 w3;  w2 = J2^T nu2;  nu1 = dt/6 l + dt/2 w2;  w1 = J1^T nu1
    l_n = l + w1 + w2 + w3 + w4,   J_i = dR/dU at the stage input y_i.
Stage inputs are recomputed from checkpoints stored every `every` steps.

Objective (not in the paper): K(U) = sum_e sum_rho w_rho J_rho |m|^2 / (2 rho),
the volume-integrated kinetic energy by solution-point quadrature.
"""

from __future__ import annotations

import numpy as np

from . import physics as ph
from .system import FRSystem, EULER

H_CS = 1e-30          # complex-step size


def _local_jac_T(fun, u, a, nin):
    """(d fun / d u)^T a for fun: R^nin -> R^nout applied column-wise.

    u: [nin, npts] (real), a: [nout, npts]; exact by complex step."""
    out = np.zeros_like(u, dtype=np.float64)
    for k in range(nin):
        du = np.zeros(u.shape, complex)
        du[k] = 1j * H_CS
        col = fun(u + du).imag / H_CS             # [nout, npts] = d fun / d u_k
        out[k] = np.sum(col * a, axis=0)
    return out


class EulerAdjoint:
    """Adjoint of ``FRSystem.rhs`` (Euler only) and of ``FRSystem.rk4``."""

    def __init__(self, sysm: FRSystem):
        if sysm.system != EULER:
            raise ValueError("the adjoint covers the Euler equations")
        self.s = sysm

    # ----------------------------------------------------------- RHS
    def rhs_vjp(self, U, lam):
        """(dR/dU)^T lam for per-block arrays [nupts, nvars, nelem]."""
        s = self.s
        prm = s.prm
        gamma = prm["gamma"]
        d, V = s.ndims, s.nvars
        P, B = s.pairs, s.bpairs
        mu = [-l / g["det"].T[:, None, :] for l, g in zip(lam, s.geo)]
        gD = [np.einsum("uf,uvn->fvn", el.M3, m) for el, m in zip(s.eles, mu)]
        gF = [np.einsum("ua,uvn->avn", el.M1, m) - np.einsum("fa,fvn->avn", el.M2, gd)
              for el, m, gd in zip(s.eles, mu, gD)]
        # point-wise transformed flux: F~_i = sum_j adj_ij f_j(u)
        out = []
        for b, (el, g, u, gf) in enumerate(zip(s.eles, s.geo, U, gF)):
            nu = el.nupts
            gfi = gf.reshape(d, nu, V, -1)                              # [i, sigma, alpha, n]
            G = np.einsum("nuij,iuvn->juvn", g["adj"], gfi)             # adj^T g: [j, sigma, alpha, n]
            ua = u.transpose(1, 0, 2).reshape(V, -1)                    # [V, nu*nel]
            Ga = G.transpose(0, 2, 1, 3).reshape(d * V, -1)             # [(j, alpha), nu*nel]
            flux = lambda w: ph.inviscid_flux(w, gamma).reshape(d * V, -1)
            au = _local_jac_T(flux, ua, Ga, V).reshape(V, nu, -1).transpose(1, 0, 2)
            out.append(au)
        # interface pairs
        uf = [np.einsum("fu,uvn->fvn", el.M0, u) for el, u in zip(s.eles, U)]
        auf = [np.zeros_like(x) for x in uf]
        uL = s._gather(uf, P["bL"], P["fL"], P["nL"])
        uR = s._gather(uf, P["bR"], P["fR"], P["nR"])
        a = P["magL"] * s._gather(gD, P["bL"], P["fL"], P["nL"]) - P["magR"] * s._gather(gD, P["bR"], P["fR"], P["nR"])
        n = P["nrm"]
        aL = _local_jac_T(lambda w: ph.rusanov(w, uR, n, gamma), uL, a, V)
        aR = _local_jac_T(lambda w: ph.rusanov(uL, w, n, gamma), uR, a, V)
        s._scatter(auf, P["bL"], P["fL"], P["nL"], aL)
        s._scatter(auf, P["bR"], P["fR"], P["nR"], aR)
        if len(B["b"]):
            ub = s._gather(uf, B["b"], B["f"], B["n"])
            ab = B["mag"] * s._gather(gD, B["b"], B["f"], B["n"])
            res = np.zeros_like(ub)
            for t in np.unique(B["t"]):
                m = B["t"] == t
                nb = B["nrm"][:, m]

                def fb(w, t=int(t), nb=nb):
                    gi, _, _ = ph.ghost_states(t, w, None, prm)
                    return ph.rusanov(w, gi, nb, gamma)
                res[:, m] = _local_jac_T(fb, ub[:, m], ab[:, m], V)
            s._scatter(auf, B["b"], B["f"], B["n"], res)
        for b, el in enumerate(s.eles):
            out[b] = out[b] + np.einsum("fu,fvn->uvn", el.M0, auf[b])
        return out

    def rhs_jvp(self, U, dU):
        """(dR/dU) dU by complex step (exact to round-off)."""
        Z = [u + 1j * H_CS * du for u, du in zip(U, dU)]
        return [r.imag / H_CS for r in self.s.rhs(Z)]

    # ----------------------------------------------------------- objective
    def kinetic_energy(self, U):
        tot = 0.0
        for b, u in enumerate(U):
            w = self.s.quadrature_weights(b)
            m2 = sum(u[:, 1 + i] ** 2 for i in range(self.s.ndims))
            tot += np.sum(w * 0.5 * m2 / u[:, 0])
        return tot

    def kinetic_energy_grad(self, U):
        G = []
        for b, u in enumerate(U):
            w = self.s.quadrature_weights(b)
            g = np.zeros_like(u)
            m2 = sum(u[:, 1 + i] ** 2 for i in range(self.s.ndims))
            g[:, 0] = -0.5 * w * m2 / u[:, 0] ** 2
            for i in range(self.s.ndims):
                g[:, 1 + i] = w * u[:, 1 + i] / u[:, 0]
            G.append(g)
        return G

    # ----------------------------------------------------------- RK4
    def _step_stages(self, u, dt):
        R = self.s.rhs
        y1 = u
        k1 = R(y1)
        y2 = [a + 0.5 * dt * k for a, k in zip(u, k1)]
        k2 = R(y2)
        y3 = [a + 0.5 * dt * k for a, k in zip(u, k2)]
        k3 = R(y3)
        y4 = [a + dt * k for a, k in zip(u, k3)]
        k4 = R(y4)
        un = [a + dt / 6.0 * (p + 2 * q + 2 * r + t) for a, p, q, r, t in zip(u, k1, k2, k3, k4)]
        return (y1, y2, y3, y4), un

    def rk4_vjp(self, U0, dt, nsteps, lam_N, every=10):
        """dK/dU0 given lam_N = dK/dU_N, RK4 stage inputs recomputed from
        checkpoints stored every `every` steps."""
        ck = {}
        u = [x.copy() for x in U0]
        for n in range(nsteps):
            if n % every == 0:
                ck[n] = [x.copy() for x in u]
            _, u = self._step_stages(u, dt)
        lam = [x.copy() for x in lam_N]
        for n in range(nsteps - 1, -1, -1):
            base = (n // every) * every
            u = [x.copy() for x in ck[base]]
            for _ in range(n - base):
                _, u = self._step_stages(u, dt)
            (y1, y2, y3, y4), _ = self._step_stages(u, dt)
            V = self.rhs_vjp
            w4 = V(y4, [dt / 6.0 * l for l in lam])
            w3 = V(y3, [dt / 3.0 * l + dt * w for l, w in zip(lam, w4)])
            w2 = V(y2, [dt / 3.0 * l + 0.5 * dt * w for l, w in zip(lam, w3)])
            w1 = V(y1, [dt / 6.0 * l + 0.5 * dt * w for l, w in zip(lam, w2)])
            lam = [l + a + b + c + e for l, a, b, c, e in zip(lam, w1, w2, w3, w4)]
        return lam
