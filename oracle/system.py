"""The FR semi-discretisation assembled on a mesh: dU/dt = R(U) (Sec. 2, App. A).

Steps, in the paper's order (Fig. flow, App. A), for every element type e:

1. U^(f) = M0 U^(u)                                    (Eq. ufpts / ufptsm)
2. Navier-Stokes only: common solution C at every flux-point pair (Eq.
   commsoln, LDG form of Sec. 4.3; boundary ghosts of App. C), then
   Q~ = M6 {C - U^(f)} + M4 U^(u)                     (Eq. transqu / tquptsm)
   Q  = J^{-T} Q~ at solution points, Q^(f) = M5 Q      (Eq. gradufpts)
3. F~ = J J^{-1} f(U, Q) at solution points (transformed flux, Sec. 2)
4. common normal flux at every pair (Eq. commpflux): Rusanov (App. B) minus the
   LDG viscous flux (Sec. 4.3), scaled by J^(f) n^(f) on each side with
   opposite signs
5. R~ = M3 {D~ - M2 F~} + M1 F~                        (Eq. tdivflux, App. A)
6. R = -J^{-1} R~                                      (Eq. negdivconf)

Readings (paper silent or ambiguous):

* Flux-point pairs are found by physical coordinates (Sec. 2 requires the two
  points of a pair to coincide), trying every combination of the periodic
  translations.  The L side of a pair is the one whose (block, element, face)
  is lexicographically smaller; each pair is visited once.
* LDG penalty sign: the common flux is
  F = F_inv - n_L.{(1/2+b) fv_L + (1/2-b) fv_R} + tau (u_L - u_R), i.e. tau
  acts as a dissipative penalty (as printed, F_vis contains +tau(u_L-u_R) and
  F = F_inv - F_vis, which would be anti-dissipative).
* Boundary: C = C(u_L, B_ldg u_L); F uses B_inv u_L in the Rusanov part and
  (B_ldg u_L, B q_L) in the LDG part (App. C allows distinct ghosts).
"""

from __future__ import annotations

import itertools

import numpy as np
from scipy.spatial import cKDTree

from .elements import RefElement
from .geometry import solution_point_metrics, flux_point_metrics
from . import physics as ph

EULER, NAVIER_STOKES = "euler", "ns"

DEFAULTS = dict(gamma=1.4, mu=0.0, prandtl=0.72, ldg_beta=0.5, ldg_tau=0.1,
                bc_rho=1.0, bc_v=(1.0, 0.0, 0.0), bc_p=1.0, outflow_p=1.0,
                wall_cpTw=1.0, wall_v=(0.0, 0.0, 0.0), wall2_v=(0.0, 0.0, 0.0))


class FRSystem:
    """Plain FP64 FR right-hand side on a ``fr_inputs.Mesh``."""

    def __init__(self, mesh, order: int, system: str = EULER, **params):
        self.mesh = mesh
        self.p = order
        self.system = system
        self.prm = dict(DEFAULTS)
        self.prm.update(params)
        self.ndims = mesh.ndims
        self.nvars = self.ndims + 2
        self.correction = self.prm.pop("correction", "dg")
        self.eles = [RefElement(b.etype, order, self.correction) for b in mesh.blocks]
        self.geo = []
        for b, el in zip(mesh.blocks, self.eles):
            Xu, det, adj = solution_point_metrics(b.etype, b.nodes, el.upts)
            Xf, mag, nrm, detf = flux_point_metrics(b.etype, b.nodes, el.fpts, el.fnorm)
            if np.any(det <= 0.0) or np.any(detf <= 0.0):
                raise ValueError("non-positive Jacobian")
            self.geo.append(dict(Xu=Xu, det=det, adj=adj, Xf=Xf, mag=mag, nrm=nrm))
        self._pair()

    # ------------------------------------------------------------ pairing
    def _pair(self):
        d = self.ndims
        X, blk, ele, fpt = [], [], [], []
        for b, (el, g) in enumerate(zip(self.eles, self.geo)):
            nel = g["Xf"].shape[0]
            X.append(g["Xf"].reshape(-1, d))
            blk.append(np.full(nel * el.nfpts, b))
            ele.append(np.repeat(np.arange(nel), el.nfpts))
            fpt.append(np.tile(np.arange(el.nfpts), nel))
        X = np.concatenate(X)
        blk, ele, fpt = (np.concatenate(a) for a in (blk, ele, fpt))
        face = np.empty_like(fpt)
        for b, el in enumerate(self.eles):
            m = blk == b
            face[m] = el.fface[fpt[m]]
        ext = np.ptp(X, axis=0).max() if len(X) else 1.0
        tol = 1e-8 * max(ext, 1.0)
        tree = cKDTree(X)
        per = np.asarray(self.mesh.periodic, np.float64).reshape(-1, d)
        shifts = [sum((k * s for k, s in zip(ks, per)), np.zeros(d))
                  for ks in itertools.product((-1, 0, 1), repeat=len(per))]
        partner = np.full(len(X), -1)
        for sh in shifts:
            hits = tree.query_ball_point(X + sh, tol)
            for i, h in enumerate(hits):
                for j in h:
                    if j == i:
                        continue
                    if partner[i] not in (-1, j):
                        raise ValueError("flux point matched twice")
                    partner[i] = j
        # boundary flux points
        btype = np.full(len(X), -1)
        offs = np.cumsum([0] + [g["Xf"].shape[0] * el.nfpts for el, g in zip(self.eles, self.geo)])
        for (b, e, f, t) in np.asarray(self.mesh.bfaces).reshape(-1, 4):
            el = self.eles[b]
            ids = offs[b] + e * el.nfpts + el.face_fpts[f]
            btype[ids] = t
        if np.any((partner < 0) & (btype < 0)):
            raise ValueError("unmatched flux point")
        if np.any((partner >= 0) & (btype >= 0)):
            raise ValueError("boundary flux point also paired")
        i = np.nonzero(partner >= 0)[0]
        j = partner[i]
        if np.any(partner[j] != i):
            raise ValueError("asymmetric pairing")
        keyi = np.stack([blk[i], ele[i], face[i]], 1)
        keyj = np.stack([blk[j], ele[j], face[j]], 1)
        # L side = lexicographically smaller (block, element, face)
        smaller = np.array([tuple(a) < tuple(b) for a, b in zip(keyi, keyj)], dtype=bool)
        L, R = i[smaller], j[smaller]
        self.pairs = dict(bL=blk[L], fL=fpt[L], nL=ele[L], bR=blk[R], fR=fpt[R], nR=ele[R])
        nrm = np.empty((len(L), d))
        magL = np.empty(len(L))
        magR = np.empty(len(L))
        for k, (bl, fl, nl, br, fr, nr) in enumerate(zip(*(self.pairs[x] for x in ("bL", "fL", "nL", "bR", "fR", "nR")))):
            nrm[k] = self.geo[bl]["nrm"][nl, fl]
            magL[k] = self.geo[bl]["mag"][nl, fl]
            magR[k] = self.geo[br]["mag"][nr, fr]
        self.pairs.update(nrm=nrm.T.copy(), magL=magL, magR=magR)
        bi = np.nonzero(btype >= 0)[0]
        self.bpairs = dict(b=blk[bi], f=fpt[bi], n=ele[bi], t=btype[bi])
        bn = np.array([self.geo[b]["nrm"][n, f] for b, f, n in zip(blk[bi], fpt[bi], ele[bi])]).reshape(-1, d)
        bm = np.array([self.geo[b]["mag"][n, f] for b, f, n in zip(blk[bi], fpt[bi], ele[bi])])
        self.bpairs.update(nrm=bn.T.copy(), mag=bm)

    # ------------------------------------------------------------ helpers
    def solution_coords(self, b):
        """Physical coordinates of solution points as [ndims, nupts, nelem]."""
        return self.geo[b]["Xu"].transpose(2, 1, 0).copy()

    def _gather(self, arrs, b, f, n):
        """Values at flux points (b, f, n) from per-block [nf, V, nel] arrays -> [V, np]."""
        out = np.empty((arrs[0].shape[-2], len(b)), dtype=arrs[0].dtype)
        for bb in np.unique(b):
            m = b == bb
            out[:, m] = arrs[bb][f[m], :, n[m]].T
        return out

    def _gather_grad(self, arrs, b, f, n):
        """Gradient values from per-block [d, nf, V, nel] arrays -> [d, V, np]."""
        d = self.ndims
        out = np.empty((d, arrs[0].shape[-2], len(b)), dtype=arrs[0].dtype)
        for bb in np.unique(b):
            m = b == bb
            out[:, :, m] = arrs[bb][:, f[m], :, n[m]].transpose(1, 2, 0)
        return out

    def _scatter(self, arrs, b, f, n, vals):
        for bb in np.unique(b):
            m = b == bb
            arrs[bb][f[m], :, n[m]] = vals[:, m].T

    # ------------------------------------------------------------ RHS
    def gradients(self, U):
        """Steps 1-2: U^(f) per block ([nfpts, V, nelem]) and, for
        Navier-Stokes, the physical gradient Q at solution points
        ([d, nupts, V, nelem]) and Q^(f) at flux points ([d, nfpts, V, nelem]);
        Q and Q^(f) are None for the Euler equations."""
        beta = self.prm["ldg_beta"]
        d, V = self.ndims, self.nvars
        P, B = self.pairs, self.bpairs
        # 1. interpolate to flux points
        Uf = [np.einsum("fu,uvn->fvn", el.M0, u) for el, u in zip(self.eles, U)]
        if self.system != NAVIER_STOKES:
            return Uf, None, None
        uL = self._gather(Uf, P["bL"], P["fL"], P["nL"])
        uR = self._gather(Uf, P["bR"], P["fR"], P["nR"])
        ub = self._gather(Uf, B["b"], B["f"], B["n"])
        # 2a. common solution (each pair visited once, both sides get it)
        C = [np.empty_like(u) for u in Uf]
        c = ph.ldg_common_solution(uL, uR, beta)
        self._scatter(C, P["bL"], P["fL"], P["nL"], c)
        self._scatter(C, P["bR"], P["fR"], P["nR"], c)
        cb = np.empty_like(ub)
        for t in np.unique(B["t"]):
            m = B["t"] == t
            _, gl, _ = ph.ghost_states(int(t), ub[:, m], None, self.prm)
            cb[:, m] = ph.ldg_common_solution(ub[:, m], gl, beta)
        self._scatter(C, B["b"], B["f"], B["n"], cb)
        # 2b. corrected transformed gradient, physical gradient, to flux points
        Q, Qf = [], []
        for el, g, u, uf, cf in zip(self.eles, self.geo, U, Uf, C):
            nu = el.nupts
            qt = (np.einsum("af,fvn->avn", el.M6, cf - uf)
                  + np.einsum("au,uvn->avn", el.M4, u)).reshape(d, nu, V, -1)
            # q_j = sum_i (J^{-1})_{ij} qt_i with J^{-1} = adj / det
            q = np.einsum("nuij,iuvn->juvn", g["adj"], qt) / g["det"].T[None, :, None, :]
            Q.append(q)
            Qf.append(np.einsum("fu,juvn->jfvn", el.M0, q))
        return Uf, Q, Qf

    def rhs(self, U, scale=False):
        """R(U) for a list of per-block states U_b[nupts, nvars, nelem].

        With scale=True also returns, per block, the magnitude
        S = |J^{-1}| (|M3| |D~| + |M3| |M2| |F~| + |M1| |F~|) of the terms whose
        sum is R (step 5 below): the componentwise forward-error scale of the
        final contraction, |R_computed - R| <= c eps S for a computation with
        unit round-off eps in its last stages.
        """
        prm = self.prm
        gamma, beta, tau = prm["gamma"], prm["ldg_beta"], prm["ldg_tau"]
        mu, pr = prm["mu"], prm["prandtl"]
        ns = self.system == NAVIER_STOKES
        d, V = self.ndims, self.nvars
        P, B = self.pairs, self.bpairs
        # 1.-2. flux-point values and (Navier-Stokes) gradients
        Uf, Q, Qf = self.gradients(U)
        uL = self._gather(Uf, P["bL"], P["fL"], P["nL"])
        uR = self._gather(Uf, P["bR"], P["fR"], P["nR"])
        ub = self._gather(Uf, B["b"], B["f"], B["n"])
        # 3. transformed flux at solution points
        Ft = []
        for b, (el, g, u) in enumerate(zip(self.eles, self.geo, U)):
            ua = u.transpose(1, 0, 2)                                  # [V, nu, nel]
            f = ph.inviscid_flux(ua, gamma)                            # [d, V, nu, nel]
            if ns:
                qa = Q[b].transpose(0, 2, 1, 3)                        # [d, V, nu, nel]
                f = f - ph.viscous_flux(ua, qa, gamma, mu, pr)
            ft = np.einsum("nuij,jvun->iuvn", g["adj"], f)              # [d, nu, V, nel]
            Ft.append(ft.reshape(d * el.nupts, V, -1))
        # 4. common normal flux at pairs and boundaries
        n = P["nrm"]
        F = ph.rusanov(uL, uR, n, gamma)
        if ns:
            qL = self._gather_grad(Qf, P["bL"], P["fL"], P["nL"])
            qR = self._gather_grad(Qf, P["bR"], P["fR"], P["nR"])
            fvL = ph.viscous_flux(uL, qL, gamma, mu, pr)
            fvR = ph.viscous_flux(uR, qR, gamma, mu, pr)
            F = F - ph.ldg_viscous_normal(fvL, fvR, n, beta) + tau * (uL - uR)
        D = [np.empty_like(u) for u in Uf]
        self._scatter(D, P["bL"], P["fL"], P["nL"], P["magL"] * F)
        self._scatter(D, P["bR"], P["fR"], P["nR"], -P["magR"] * F)
        if len(B["b"]):
            Fb = np.empty_like(ub)
            qb = self._gather_grad(Qf, B["b"], B["f"], B["n"]) if ns else None
            for t in np.unique(B["t"]):
                m = B["t"] == t
                gi, gl, qg = ph.ghost_states(int(t), ub[:, m], None if qb is None else qb[:, :, m], prm)
                nb = B["nrm"][:, m]
                Fm = ph.rusanov(ub[:, m], gi, nb, gamma)
                if ns:
                    fvL = ph.viscous_flux(ub[:, m], qb[:, :, m], gamma, mu, pr)
                    fvR = ph.viscous_flux(gl, qg, gamma, mu, pr)
                    Fm = Fm - ph.ldg_viscous_normal(fvL, fvR, nb, beta) + tau * (ub[:, m] - gl)
                Fb[:, m] = Fm
            self._scatter(D, B["b"], B["f"], B["n"], B["mag"] * Fb)
        # 5./6. corrected divergence and negation
        R, S = [], []
        for el, g, dd, ft in zip(self.eles, self.geo, D, Ft):
            rt = (np.einsum("uf,fvn->uvn", el.M3, dd - np.einsum("fa,avn->fvn", el.M2, ft))
                  + np.einsum("ua,avn->uvn", el.M1, ft))
            R.append(-rt / g["det"].T[:, None, :])
            if scale:
                aM3, aM2, aM1 = np.abs(el.M3), np.abs(el.M2), np.abs(el.M1)
                aD, aF = np.abs(dd), np.abs(ft)
                st = (np.einsum("uf,fvn->uvn", aM3, aD + np.einsum("fa,avn->fvn", aM2, aF))
                      + np.einsum("ua,avn->uvn", aM1, aF))
                S.append(st / np.abs(g["det"]).T[:, None, :])
        return (R, S) if scale else R

    # ------------------------------------------------------------ time stepping
    def rk4(self, U, dt, nsteps=1):
        """Classical RK4 (Sec. 2 end; Sec. 5.1)."""
        U = [u.copy() for u in U]
        for _ in range(nsteps):
            k1 = self.rhs(U)
            k2 = self.rhs([u + 0.5 * dt * k for u, k in zip(U, k1)])
            k3 = self.rhs([u + 0.5 * dt * k for u, k in zip(U, k2)])
            k4 = self.rhs([u + dt * k for u, k in zip(U, k3)])
            U = [u + dt / 6.0 * (a + 2.0 * b + 2.0 * c + e)
                 for u, a, b, c, e in zip(U, k1, k2, k3, k4)]
        return U

    def euler(self, U, dt, nsteps=1):
        """Forward Euler (Sec. 3)."""
        from .steppers import euler
        return euler(self.rhs, U, dt, nsteps)

    def dopri5(self, U, dt, nsteps=1, atol=1e-6, rtol=1e-6):
        """nsteps fixed DOPRI5 steps (Sec. 3); returns (U, error norm of the last step)."""
        from .steppers import dopri5
        return dopri5(self.rhs, U, dt, nsteps, atol, rtol)

    # ------------------------------------------------------------ diagnostics
    def quadrature_weights(self, b):
        """w_rho J_rho at solution points ([nupts, nelem]): the solution-point
        quadrature used for the conservation sum (exact for tensor GL points)."""
        el = self.eles[b]
        if el.etype in ("quad", "hex"):
            from .polys import gauss_legendre
            _, w1 = gauss_legendre(el.p + 1)
            w = w1
            for _ in range(el.ndims - 1):
                w = np.outer(w1, w).ravel()
        else:
            # weights of the interpolatory rule on the solution points
            xq, wq = el.volume_quadrature(el.p + 2)
            w = el.nodal(xq) @ wq
        return w[:, None] * self.geo[b]["det"].T
