"""Standard elements, nodal bases and the constant operator matrices M0..M6.

Follows Sec. 2 (solution/flux points, nodal basis through the generalised
Vandermonde matrix, correction functions constrained by Eq. corfn) and
App. A (operator matrices).  Readings of the paper used here:

* Reference elements and point orderings (paper silent): quad [-1,1]^2 and hex
  [-1,1]^3 with tensor Gauss-Legendre solution points, xi fastest; triangle
  with vertices (-1,-1), (1,-1), (-1,1).  Faces and face-point orderings are
  listed in ``FACES``.
* Triangle solution points: the Williams-Shunn coordinates of Sec. 5.2 are not
  in the paper; the interior nodes of the degree-(p+3) equispaced lattice
  (an affine image of the degree-p principal lattice, hence unisolvent for
  P_p) are used instead.  Flux points are Gauss-Legendre on every edge.
* DG correction functions (Sec. 5.1 names "DG" only): div g_sigma is the
  P_p (triangle) / Q_p (tensor element) lift of the face Lagrange polynomial of
  flux point sigma, i.e. int(phi_sigma v) = surface-int(l_sigma v) for all v in
  the solution space, with the exact mass matrix and reference arc length /
  face area.
* SD and HU correction functions (Sec. 5.1 runs DG, SD and HU "as defined in"
  Vincent, Castonguay and Jameson 2011, whose formulas the paper does not
  print): the one-parameter VCJH family in 1D,
      g_R = (P_p + (eta P_{p-1} + P_{p+1}) / (1 + eta)) / 2,
      eta = c (2p+1) (a_p p!)^2 / 2,  a_p = (2p)! / (2^p (p!)^2),
  with c_DG = 0, c_SD = 2p / ((2p+1)(p+1)(a_p p!)^2) and
  c_HU = 2(p+1) / ((2p+1) p (a_p p!)^2), i.e. eta = 0, p/(p+1), (p+1)/p; on a
  tensor element div g_sigma = g_R'(s xi_n) times the 1D Lagrange factors of
  sigma's tangential coordinates (xi_n the coordinate normal to sigma's face,
  s its outward sign).  Triangles: DG only (the simplex VCJH construction is
  a separate paper the source does not summarise).
* M6 as printed in App. A is garbled; it is read as
  (M6)_{(i sigma), rho} = n_{rho,i} (div g_rho)(x_sigma^(u)), which makes
  Eq. tquptsm reproduce Eq. transqu with component stride N^(u).
"""

from __future__ import annotations

import numpy as np

from .polys import gauss_legendre, legendre, jacobi, lagrange

NDIMS = {"quad": 2, "tri": 2, "hex": 3}
# VCJH parameter eta(p) of the named correction functions (Vincent et al. 2011)
VCJH_ETA = {"dg": lambda p: 0.0, "sd": lambda p: p / (p + 1.0), "hu": lambda p: (p + 1.0) / p}


def vcjh_right(p, correction, x):
    """Right VCJH correction function g_R and its derivative at x."""
    eta = VCJH_ETA[correction](p)
    lp, dp = legendre(p, x)
    lm, dm = legendre(p - 1, x) if p >= 1 else (np.zeros_like(lp), np.zeros_like(lp))
    l1, d1 = legendre(p + 1, x)
    g = 0.5 * (lp + (eta * lm + l1) / (1.0 + eta))
    dg = 0.5 * (dp + (eta * dm + d1) / (1.0 + eta))
    return g, dg
NFACES = {"quad": 4, "tri": 3, "hex": 6}


def _face_maps(etype):
    """Per face: (map from face parameters to reference coords, unit normal,
    reference surface measure per unit parameter measure)."""
    s2 = np.sqrt(2.0)
    if etype == "quad":
        return [
            (lambda t: np.stack([t, -np.ones_like(t)]), np.array([0.0, -1.0]), 1.0),
            (lambda t: np.stack([np.ones_like(t), t]), np.array([1.0, 0.0]), 1.0),
            (lambda t: np.stack([-t, np.ones_like(t)]), np.array([0.0, 1.0]), 1.0),
            (lambda t: np.stack([-np.ones_like(t), -t]), np.array([-1.0, 0.0]), 1.0),
        ]
    if etype == "tri":
        return [
            (lambda t: np.stack([t, -np.ones_like(t)]), np.array([0.0, -1.0]), 1.0),
            (lambda t: np.stack([-t, t]), np.array([1.0, 1.0]) / s2, s2),
            (lambda t: np.stack([-np.ones_like(t), -t]), np.array([-1.0, 0.0]), 1.0),
        ]
    if etype == "hex":
        m, p = -1.0, 1.0
        def mk(fix_axis, val):
            def f(ab):
                a, b = ab
                c = np.full_like(a, val)
                free = [ax for ax in range(3) if ax != fix_axis]
                out = [None] * 3
                out[free[0]], out[free[1]], out[fix_axis] = a, b, c
                return np.stack(out)
            return f
        n = lambda *v: np.array(v, np.float64)
        return [
            (mk(2, m), n(0, 0, -1), 1.0),
            (mk(1, m), n(0, -1, 0), 1.0),
            (mk(0, p), n(1, 0, 0), 1.0),
            (mk(1, p), n(0, 1, 0), 1.0),
            (mk(0, m), n(-1, 0, 0), 1.0),
            (mk(2, p), n(0, 0, 1), 1.0),
        ]
    raise ValueError(etype)


class RefElement:
    """Standard element of type ``etype`` at polynomial order ``p``."""

    def __init__(self, etype: str, p: int, correction: str = "dg"):
        if correction not in VCJH_ETA:
            raise ValueError(f"unknown correction {correction!r}")
        if correction != "dg" and etype == "tri":
            raise ValueError("SD / HU corrections are defined here for tensor elements only")
        self.etype, self.p = etype, p
        self.correction = correction
        self.ndims = NDIMS[etype]
        self.nfaces = NFACES[etype]
        gl, _ = gauss_legendre(p + 1)
        self.gl = gl
        # ---- solution points -------------------------------------------------
        if etype == "quad":
            xi, eta = np.meshgrid(gl, gl, indexing="xy")          # xi fastest
            self.upts = np.stack([xi.ravel(), eta.ravel()], axis=1)
        elif etype == "hex":
            zz, yy, xx = np.meshgrid(gl, gl, gl, indexing="ij")
            self.upts = np.stack([xx.ravel(), yy.ravel(), zz.ravel()], axis=1)
        else:
            pts = []
            for j in range(p + 1):
                for i in range(p + 1 - j):
                    pts.append((-1.0 + 2.0 * (i + 1) / (p + 3), -1.0 + 2.0 * (j + 1) / (p + 3)))
            self.upts = np.asarray(pts)
        self.nupts = self.upts.shape[0]
        # ---- flux points -----------------------------------------------------
        self.faces = _face_maps(etype)
        fpts, fnorm, fface = [], [], []
        self.face_fpts = []
        for f, (fmap, nrm, _) in enumerate(self.faces):
            if self.ndims == 2:
                par = gl[None, :]
            else:
                b, a = np.meshgrid(gl, gl, indexing="ij")          # a fastest
                par = np.stack([a.ravel(), b.ravel()])
            x = fmap(par[0] if self.ndims == 2 else par)
            start = len(fpts)
            for k in range(x.shape[1]):
                fpts.append(x[:, k]); fnorm.append(nrm); fface.append(f)
            self.face_fpts.append(np.arange(start, len(fpts)))
        self.fpts = np.asarray(fpts)
        self.fnorm = np.asarray(fnorm)
        self.fface = np.asarray(fface)
        self.nfpts = self.fpts.shape[0]
        # ---- nodal basis via the generalised Vandermonde matrix -------------
        self.V = self.psi(self.upts.T)                              # [nbasis, nupts]
        self._build_operators()

    def _vcjh_M3(self):
        """div g_sigma at the solution points for a tensor element: the VCJH
        g_R' along the face normal times the tangential 1D Lagrange factors."""
        d, nu, nf = self.ndims, self.nupts, self.nfpts
        M3 = np.zeros((nu, nf))
        for sg in range(nf):
            ax = int(np.argmax(np.abs(self.fnorm[sg])))
            sgn = np.sign(self.fnorm[sg, ax])
            _, dg = vcjh_right(self.p, self.correction, sgn * self.upts[:, ax])
            col = dg.copy()
            for k in range(d):
                if k == ax:
                    continue
                j = int(np.argmin(np.abs(self.gl - self.fpts[sg, k])))
                lk, _ = lagrange(self.gl, self.upts[:, k])
                col *= lk[j]
            M3[:, sg] = col
        return M3

    # --- spanning basis psi (any basis of the order-p space works, Sec. 2) ---
    def _psi_grad(self, x):
        p = self.p
        if self.etype in ("quad", "hex"):
            P = [[legendre(k, x[d]) for k in range(p + 1)] for d in range(self.ndims)]
            vals, grads = [], []
            for idx in np.ndindex(*(p + 1,) * self.ndims):
                v = np.ones_like(x[0])
                for d in range(self.ndims):
                    v = v * P[d][idx[d]][0]
                g = []
                for dd in range(self.ndims):
                    gd = np.ones_like(x[0])
                    for d in range(self.ndims):
                        gd = gd * (P[d][idx[d]][1] if d == dd else P[d][idx[d]][0])
                    g.append(gd)
                vals.append(v); grads.append(g)
            return np.asarray(vals), np.asarray(grads).transpose(1, 0, *range(2, x.ndim + 1))
        # triangle: Dubiner basis on collapsed coordinates (a, b)
        r, s = x[0], x[1]
        b = s
        a = 2.0 * (1.0 + r) / (1.0 - s) - 1.0
        vals, gr, gs = [], [], []
        for i in range(p + 1):
            Pa, dPa = legendre(i, a)
            for j in range(p + 1 - i):
                Pb, dPb = jacobi(j, 2.0 * i + 1.0, 0.0, b)
                h = ((1.0 - b) / 2.0) ** i
                dh = -0.5 * i * ((1.0 - b) / 2.0) ** (i - 1) if i > 0 else np.zeros_like(b)
                vals.append(Pa * Pb * h)
                # d/dr: da/dr = 2/(1-s)
                gr.append(dPa * 2.0 / (1.0 - s) * Pb * h)
                # d/ds: da/ds = (1+a)/(1-s), db/ds = 1
                gs.append(dPa * (1.0 + a) / (1.0 - s) * Pb * h + Pa * (dPb * h + Pb * dh))
        return np.asarray(vals), np.stack([np.asarray(gr), np.asarray(gs)])

    def psi(self, x):
        return self._psi_grad(np.asarray(x, np.float64))[0]

    def nodal(self, x):
        """l_rho(x) = sum_sigma Vinv[rho, sigma] psi_sigma(x); returns [nupts, npts].

        V[rho, sigma] = psi_rho(x_sigma^(u)) is the generalised Vandermonde
        matrix of Sec. 2, so l_rho(x_tau^(u)) = delta_{rho tau}.
        """
        ps = self.psi(x)
        Vinv = np.linalg.inv(self.V)
        return (Vinv @ ps.reshape(ps.shape[0], -1)).reshape((self.nupts,) + ps.shape[1:])

    def dnodal(self, x):
        """Gradient of the nodal basis; returns [ndims, nupts, npts]."""
        _, g = self._psi_grad(np.asarray(x, np.float64))
        Vinv = np.linalg.inv(self.V)
        return np.stack([(Vinv @ g[d].reshape(g.shape[1], -1)).reshape((self.nupts,) + g.shape[2:])
                         for d in range(self.ndims)])

    # --- quadrature on the element and its faces ------------------------------
    def volume_quadrature(self, n):
        x, w = gauss_legendre(n)
        if self.etype == "quad":
            X, Y = np.meshgrid(x, x, indexing="xy")
            W = np.outer(w, w)
            return np.stack([X.ravel(), Y.ravel()]), W.ravel()
        if self.etype == "hex":
            Z, Y, X = np.meshgrid(x, x, x, indexing="ij")
            W = w[:, None, None] * w[None, :, None] * w[None, None, :]
            return np.stack([X.ravel(), Y.ravel(), Z.ravel()]), W.ravel()
        # triangle: collapsed (Duffy) map of the square, Jacobian (1-b)/2
        A, B = np.meshgrid(x, x, indexing="xy")
        WA, WB = np.meshgrid(w, w, indexing="xy")
        r = 0.5 * (1.0 + A) * (1.0 - B) - 1.0
        s = B
        W = WA * WB * 0.5 * (1.0 - B)
        return np.stack([r.ravel(), s.ravel()]), W.ravel()

    def _build_operators(self):
        nu, nf, d = self.nupts, self.nfpts, self.ndims
        # M0: interpolation to flux points (Eq. ufpts / App. A)
        Lf = self.nodal(self.fpts.T)                               # [nu, nf]
        self.M0 = Lf.T.copy()
        # M4 / M1: nodal-basis gradients at solution points
        dL = self.dnodal(self.upts.T)                              # [d, nu(rho), nu(sigma)]
        self.M4 = dL.transpose(0, 2, 1).reshape(d * nu, nu)
        self.M1 = dL.transpose(2, 0, 1).reshape(nu, d * nu)
        # M2: interpolated flux dotted with the reference normal at flux points
        self.M2 = (self.M0[:, None, :] * self.fnorm[:, :, None]).reshape(nf, d * nu)
        # M3: divergence of the DG correction functions at solution points
        xq, wq = self.volume_quadrature(self.p + 2)
        Lq = self.nodal(xq)                                        # [nu, nq]
        mass = (Lq * wq) @ Lq.T
        E = np.zeros((nu, nf))
        tq, wt = gauss_legendre(self.p + 2)
        for f, (fmap, _, dsdt) in enumerate(self.faces):
            ids = self.face_fpts[f]
            if d == 2:
                xf = fmap(tq)
                lf, _ = lagrange(self.gl, tq)                      # [p+1, nq]
                w = wt * dsdt
            else:
                B, A = np.meshgrid(tq, tq, indexing="ij")
                WB, WA = np.meshgrid(wt, wt, indexing="ij")
                a, b = A.ravel(), B.ravel()
                xf = fmap(np.stack([a, b]))
                la, _ = lagrange(self.gl, a)
                lb, _ = lagrange(self.gl, b)
                lf = np.stack([la[i] * lb[j] for j in range(self.p + 1) for i in range(self.p + 1)])
                w = (WA * WB).ravel() * dsdt
            Lface = self.nodal(xf)                                 # [nu, nq]
            E[:, ids] = (Lface * w) @ lf.T
        self.mass = mass
        self.M3 = np.linalg.solve(mass, E)                         # [nu, nf]
        if self.correction != "dg":
            self.M3 = self._vcjh_M3()
        # M6 (reading): (M6)_{(i sigma), rho} = n_{rho,i} M3[sigma, rho]
        self.M6 = (self.fnorm.T[:, None, :] * self.M3[None, :, :]).reshape(d * nu, nf)
