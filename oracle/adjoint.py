"""Discrete adjoint of the FR right-hand side (Euler and Navier-Stokes) and of
classical RK4 (FP64).  Test infrastructure: only the tests, the smoke check
and the benchmark's CPU baseline use it.

Not in the paper: the transpose (dR/dU)^T lambda of the FR operator of
Sec. 2 / App. A, assembled by running the RHS steps backwards.  Forward map:

    uf = M0 U
    (NS)  C = LDG common solution of uf (Sec. 4.3; boundary ghosts, App. C)
          qt = M6 (C - uf) + M4 U,  Q = J^-T qt,  Qf = M0 Q (per direction)
    F~ = adj(J) (f_inv(U) - f_vis(U, Q))
    D~_L = |n|_L F(uL, uR, qL, qR, n),  D~_R = -|n|_R F(...)
    R = -J^-1 [M3 D~ + (M1 - M3 M2) F~]

Transpose:

    mu   = -J^-1 lambda
    g_D  = M3^T mu,  g_F = (M1 - M3 M2)^T mu  (= M1^T mu - M2^T g_D)
    per pair:  a = |n|_L g_D,L - |n|_R g_D,R;  a_uL, a_uR, a_qL, a_qR = (dF/d.)^T a
    boundary:  a_ub, a_qb = (d F(ub, ghosts(ub, qb)) / d.)^T (|n| g_D)
    point-wise: G = adj(J)^T g_F;  a_U = (df/dU)^T G,  a_Q = (df/dQ)^T G
    (NS)  a_Q += M0^T a_Qf;  a_qt = J^-1 a_Q (per point: adj(J) a_Q / det J)
          a_C = M6^T a_qt;  a_uf -= a_C;  a_U += M4^T a_qt
          a_uf += (dC/d uf)^T a_C   (both sides of a pair share C)
    a_U += M0^T a_uf

The local Jacobians (fluxes, the Rusanov / LDG common flux with its ghost
states, the boundary common solution) are taken exactly by the complex-step
method on the oracle's own complex-safe physics.

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
from .system import FRSystem, NAVIER_STOKES

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


def _scatter_grad(s, arrs, b, f, n, vals):
    """Write gradient values [d, V, np] at flux points (b, f, n) into per-block
    [d, nf, V, nel] arrays."""
    for bb in np.unique(b):
        m = b == bb
        arrs[bb][:, f[m], :, n[m]] = vals[:, :, m].transpose(2, 0, 1)


class FRAdjoint:
    """Adjoint of ``FRSystem.rhs`` and of ``FRSystem.rk4``."""

    def __init__(self, sysm: FRSystem):
        self.s = sysm

    # ----------------------------------------------------------- RHS
    def rhs_vjp(self, U, lam):
        """(dR/dU)^T lam for per-block arrays [nupts, nvars, nelem]."""
        s = self.s
        prm = s.prm
        gamma, beta, tau = prm["gamma"], prm["ldg_beta"], prm["ldg_tau"]
        mu, pr = prm["mu"], prm["prandtl"]
        ns = s.system == NAVIER_STOKES
        d, V = s.ndims, s.nvars
        P, B = s.pairs, s.bpairs
        Uf, Q, Qf = s.gradients(U)
        mu_ = [-l / g["det"].T[:, None, :] for l, g in zip(lam, s.geo)]
        gD = [np.einsum("uf,uvn->fvn", el.M3, m) for el, m in zip(s.eles, mu_)]
        gF = [np.einsum("ua,uvn->avn", el.M1, m) - np.einsum("fa,fvn->avn", el.M2, gd)
              for el, m, gd in zip(s.eles, mu_, gD)]

        def vflux(w, q):
            return ph.viscous_flux(w, q, gamma, mu, pr)

        # point-wise transformed flux: F~_i = sum_j adj_ij f_j(u, q)
        out, aQ = [], []
        for b, (el, g, u, gf) in enumerate(zip(s.eles, s.geo, U, gF)):
            nu = el.nupts
            gfi = gf.reshape(d, nu, V, -1)                              # [i, sigma, alpha, n]
            G = np.einsum("nuij,iuvn->juvn", g["adj"], gfi)             # adj^T g: [j, sigma, alpha, n]
            ua = u.transpose(1, 0, 2).reshape(V, -1)                    # [V, nu*nel]
            Ga = G.transpose(0, 2, 1, 3).reshape(d * V, -1)             # [(j, alpha), nu*nel]
            if ns:
                qa = Q[b].transpose(0, 2, 1, 3).reshape(d * V, -1)      # [(j, alpha), nu*nel]

                def flux(w, q):
                    f = ph.inviscid_flux(w, gamma) - vflux(w, q.reshape(d, V, -1))
                    return f.reshape(d * V, -1)
                au = _local_jac_T(lambda w: flux(w, qa), ua, Ga, V)
                aq = _local_jac_T(lambda w: flux(ua, w), qa, Ga, d * V)
                aQ.append(aq.reshape(d, V, nu, -1).transpose(0, 2, 1, 3))     # [j, sigma, alpha, n]
            else:
                au = _local_jac_T(lambda w: ph.inviscid_flux(w, gamma).reshape(d * V, -1), ua, Ga, V)
            out.append(au.reshape(V, nu, -1).transpose(1, 0, 2))
        # interface pairs
        auf = [np.zeros_like(x) for x in Uf]
        aQf = [np.zeros_like(x) for x in Qf] if ns else None
        uL = s._gather(Uf, P["bL"], P["fL"], P["nL"])
        uR = s._gather(Uf, P["bR"], P["fR"], P["nR"])
        a = P["magL"] * s._gather(gD, P["bL"], P["fL"], P["nL"]) - P["magR"] * s._gather(gD, P["bR"], P["fR"], P["nR"])
        n = P["nrm"]
        if ns:
            qL = s._gather_grad(Qf, P["bL"], P["fL"], P["nL"])
            qR = s._gather_grad(Qf, P["bR"], P["fR"], P["nR"])

            def Fp(wL, wR, zL, zR):
                return (ph.rusanov(wL, wR, n, gamma)
                        - ph.ldg_viscous_normal(vflux(wL, zL), vflux(wR, zR), n, beta) + tau * (wL - wR))
            aL = _local_jac_T(lambda w: Fp(w, uR, qL, qR), uL, a, V)
            aR = _local_jac_T(lambda w: Fp(uL, w, qL, qR), uR, a, V)
            aqL = _local_jac_T(lambda w: Fp(uL, uR, w.reshape(d, V, -1), qR), qL.reshape(d * V, -1), a, d * V)
            aqR = _local_jac_T(lambda w: Fp(uL, uR, qL, w.reshape(d, V, -1)), qR.reshape(d * V, -1), a, d * V)
            _scatter_grad(s, aQf, P["bL"], P["fL"], P["nL"], aqL.reshape(d, V, -1))
            _scatter_grad(s, aQf, P["bR"], P["fR"], P["nR"], aqR.reshape(d, V, -1))
        else:
            aL = _local_jac_T(lambda w: ph.rusanov(w, uR, n, gamma), uL, a, V)
            aR = _local_jac_T(lambda w: ph.rusanov(uL, w, n, gamma), uR, a, V)
        s._scatter(auf, P["bL"], P["fL"], P["nL"], aL)
        s._scatter(auf, P["bR"], P["fR"], P["nR"], aR)
        if len(B["b"]):
            ub = s._gather(Uf, B["b"], B["f"], B["n"])
            qb = s._gather_grad(Qf, B["b"], B["f"], B["n"]) if ns else None
            ab = B["mag"] * s._gather(gD, B["b"], B["f"], B["n"])
            res = np.zeros_like(ub)
            resq = np.zeros((d, V, ub.shape[1])) if ns else None
            for t in np.unique(B["t"]):
                m = B["t"] == t
                nb = B["nrm"][:, m]

                def fb(w, z, t=int(t), nb=nb):
                    gi, gl, qg = ph.ghost_states(t, w, z, prm)
                    F = ph.rusanov(w, gi, nb, gamma)
                    if ns:
                        F = F - ph.ldg_viscous_normal(vflux(w, z), vflux(gl, qg), nb, beta) + tau * (w - gl)
                    return F
                qm = qb[:, :, m] if ns else None
                res[:, m] = _local_jac_T(lambda w: fb(w, qm), ub[:, m], ab[:, m], V)
                if ns:
                    resq[:, :, m] = _local_jac_T(lambda w: fb(ub[:, m], w.reshape(d, V, -1)),
                                                 qm.reshape(d * V, -1), ab[:, m], d * V).reshape(d, V, -1)
            s._scatter(auf, B["b"], B["f"], B["n"], res)
            if ns:
                _scatter_grad(s, aQf, B["b"], B["f"], B["n"], resq)
        if ns:
            # gradient chain: Qf = M0 Q, Q = J^-T qt, qt = M6 (C - uf) + M4 U
            aC = []
            for b, (el, g) in enumerate(zip(s.eles, s.geo)):
                aq = aQ[b] + np.einsum("fu,jfvn->juvn", el.M0, aQf[b])          # [j, sigma, alpha, n]
                aqt = np.einsum("nuij,juvn->iuvn", g["adj"], aq) / g["det"].T[None, :, None, :]
                aqt = aqt.reshape(d * el.nupts, V, -1)
                ac = np.einsum("af,avn->fvn", el.M6, aqt)
                out[b] = out[b] + np.einsum("au,avn->uvn", el.M4, aqt)
                auf[b] = auf[b] - ac
                aC.append(ac)
            # common solution: both sides of a pair hold the same C
            acp = s._gather(aC, P["bL"], P["fL"], P["nL"]) + s._gather(aC, P["bR"], P["fR"], P["nR"])
            addL = [np.zeros_like(x) for x in Uf]
            addR = [np.zeros_like(x) for x in Uf]
            s._scatter(addL, P["bL"], P["fL"], P["nL"], (0.5 - beta) * acp)
            s._scatter(addR, P["bR"], P["fR"], P["nR"], (0.5 + beta) * acp)
            auf = [x + y + z for x, y, z in zip(auf, addL, addR)]
            if len(B["b"]):
                acb = s._gather(aC, B["b"], B["f"], B["n"])
                resc = np.zeros_like(ub)
                for t in np.unique(B["t"]):
                    m = B["t"] == t

                    def cb(w, t=int(t)):
                        _, gl, _ = ph.ghost_states(t, w, None, prm)
                        return ph.ldg_common_solution(w, gl, beta)
                    resc[:, m] = _local_jac_T(cb, ub[:, m], acb[:, m], V)
                addB = [np.zeros_like(x) for x in Uf]
                s._scatter(addB, B["b"], B["f"], B["n"], resc)
                auf = [x + y for x, y in zip(auf, addB)]
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
