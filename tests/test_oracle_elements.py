"""Pins for the standard elements and operator matrices (Sec. 2, App. A).

Independent constructions used here: a monomial Vandermonde for the nodal
basis, numpy's leggauss quadrature (over-integrated), the closed-form Radau
correction function for tensor elements, and a weak-form nodal DG residual.
"""
import itertools

import numpy as np
import numpy.polynomial.legendre as npleg
import pytest

from oracle.elements import RefElement

CASES = [("quad", p) for p in (1, 2, 3, 4)] + [("tri", p) for p in (1, 2, 3, 4)] + \
        [("hex", p) for p in (1, 2, 3)]


def monomial_exps(etype, p):
    if etype == "quad":
        return [(a, b) for b in range(p + 1) for a in range(p + 1)]
    if etype == "hex":
        return [(a, b, c) for c in range(p + 1) for b in range(p + 1) for a in range(p + 1)]
    return [(a, b) for b in range(p + 1) for a in range(p + 1 - b)]


def mono(exps, x):
    """m_k(x) [nb, npts] and gradients [d, nb, npts]."""
    x = np.asarray(x)
    d = x.shape[0]
    vals = np.array([np.prod([x[i] ** e[i] for i in range(d)], axis=0) for e in exps])
    grads = []
    for j in range(d):
        g = []
        for e in exps:
            t = np.ones_like(x[0])
            for i in range(d):
                if i == j:
                    t = t * (e[i] * x[i] ** max(e[i] - 1, 0) if e[i] > 0 else 0.0 * x[i])
                else:
                    t = t * x[i] ** e[i]
            g.append(t)
        grads.append(g)
    return vals, np.array(grads)


def nodal_mono(el):
    exps = monomial_exps(el.etype, el.p)
    Vm = mono(exps, el.upts.T)[0].T               # [sigma, k]
    C = np.linalg.inv(Vm)                         # l_rho = sum_k C[k, rho] m_k

    def ev(x):
        v, g = mono(exps, x)
        return C.T @ v, np.einsum("kr,dkq->drq", C, g)
    return ev


def vol_quad(etype, n):
    x, w = npleg.leggauss(n)
    if etype == "quad":
        X = np.array(list(itertools.product(x, x))).T[::-1]
        W = np.array([a * b for a, b in itertools.product(w, w)])
        return X, W
    if etype == "hex":
        X = np.array(list(itertools.product(x, x, x))).T[::-1]
        W = np.array([a * b * c for a, b, c in itertools.product(w, w, w)])
        return X, W
    pts, W = [], []
    for (a, wa), (b, wb) in itertools.product(zip(x, w), zip(x, w)):
        pts.append((0.5 * (1 + a) * (1 - b) - 1, b)); W.append(wa * wb * 0.5 * (1 - b))
    return np.array(pts).T, np.array(W)


# face geometry restated from the vertex lists of each standard element
FACE_VERTS = {
    "quad": [[(-1, -1), (1, -1)], [(1, -1), (1, 1)], [(1, 1), (-1, 1)], [(-1, 1), (-1, -1)]],
    "tri": [[(-1, -1), (1, -1)], [(1, -1), (-1, 1)], [(-1, 1), (-1, -1)]],
}
HEX_FACES = [(2, -1), (1, -1), (0, 1), (1, 1), (0, -1), (2, 1)]   # (fixed axis, value)


@pytest.mark.parametrize("etype,p", CASES)
def test_kronecker_and_row_sums(etype, p):
    el = RefElement(etype, p)
    assert np.allclose(el.nodal(el.upts.T), np.eye(el.nupts), atol=1e-13)
    assert np.allclose(el.M0.sum(axis=1), 1.0, atol=1e-13)
    assert np.allclose(el.M4.sum(axis=1), 0.0, atol=1e-12)


@pytest.mark.parametrize("etype,p", CASES)
def test_interpolation_and_gradient_exact_on_solution_space(etype, p):
    el = RefElement(etype, p)
    d, nu = el.ndims, el.nupts
    for e in monomial_exps(etype, p):
        vu, gu = mono([e], el.upts.T)
        vf, _ = mono([e], el.fpts.T)
        assert np.allclose(el.M0 @ vu[0], vf[0], atol=1e-12)
        grad = (el.M4 @ vu[0]).reshape(d, nu)
        assert np.allclose(grad, gu[:, 0, :], atol=1e-11)
        assert np.allclose(el.M1 @ np.concatenate([gu[i, 0] * 0 + (i == 0) * vu[0] for i in range(d)]),
                           gu[0, 0], atol=1e-11)


def radau_right_derivative(p, x):
    """g_R = (P_p + P_{p+1}) / 2: the right Radau (DG) correction function."""
    c = np.zeros(p + 2); c[p] = 0.5; c[p + 1] = 0.5
    return npleg.legval(x, npleg.legder(c))


@pytest.mark.parametrize("etype,p", [(e, p) for e, p in CASES if e != "tri"])
def test_dg_correction_matches_radau_closed_form(etype, p):
    el = RefElement(etype, p)
    d = el.ndims
    for s in range(el.nfpts):
        n = el.fnorm[s]
        ax = int(np.argmax(np.abs(n)))
        sgn = np.sign(n[ax])
        expect = np.empty(el.nupts)
        for r in range(el.nupts):
            x = el.upts[r]
            # g_sigma = n g_R(sgn xi) along the face normal, so div g = g_R'(sgn xi)
            g = radau_right_derivative(p, sgn * x[ax])
            tang = 1.0
            for k in range(d):
                if k == ax:
                    continue
                # tangential Lagrange factor: 1 where the solution point shares
                # the flux point's tangential coordinate, 0 otherwise
                tang *= float(abs(x[k] - el.fpts[s, k]) < 1e-12)
            expect[r] = g * tang
        assert np.allclose(el.M3[:, s], expect, atol=1e-12)


def _face_rules(etype, el, n):
    """(points [d, nq], weights incl. reference measure, face-Lagrange values of the
    face's flux points [nfp, nq], flux point ids) for every face."""
    t, w = npleg.leggauss(n)
    rules = []
    if etype in ("quad", "tri"):
        for f, (a, b) in enumerate(FACE_VERTS[etype]):
            a, b = np.array(a, float), np.array(b, float)
            X = a[:, None] + np.outer(b - a, (t + 1) / 2)
            ds = np.linalg.norm(b - a) / 2
            ids = np.nonzero(el.fface == f)[0]
            # parameter of each flux point along the edge (and check it is on the edge)
            tf = 2 * np.dot(el.fpts[ids] - a, b - a) / np.dot(b - a, b - a) - 1
            assert np.allclose(a[None] + np.outer((tf + 1) / 2, b - a), el.fpts[ids], atol=1e-14)
            Lf = np.array([[np.prod([(tt - tf[m]) / (tf[j] - tf[m]) for m in range(len(tf)) if m != j])
                            for tt in t] for j in range(len(tf))])
            rules.append((X, w * ds, Lf, ids))
        return rules
    for f, (ax, val) in enumerate(HEX_FACES):
        free = [k for k in range(3) if k != ax]
        A, B = np.meshgrid(t, t, indexing="ij")
        WA, WB = np.meshgrid(w, w, indexing="ij")
        X = np.zeros((3, A.size))
        X[free[0]], X[free[1]], X[ax] = A.ravel(), B.ravel(), val
        ids = np.nonzero(el.fface == f)[0]
        assert np.allclose(el.fpts[ids, ax], val)
        pa, pb = el.fpts[ids, free[0]], el.fpts[ids, free[1]]
        ua, ub = np.unique(pa), np.unique(pb)
        def lag(nodes, j, x):
            return np.prod([(x - nodes[m]) / (nodes[j] - nodes[m]) for m in range(len(nodes)) if m != j], axis=0)
        Lf = np.array([lag(ua, int(np.argmin(abs(ua - pa[k]))), X[free[0]]) *
                       lag(ub, int(np.argmin(abs(ub - pb[k]))), X[free[1]]) for k in range(len(ids))])
        rules.append((X, (WA * WB).ravel(), Lf, ids))
    return rules


@pytest.mark.parametrize("etype,p", CASES)
def test_fr_with_dg_correction_equals_nodal_dg(etype, p):
    """For F~ in the solution space and any D~, R~ = M3 (D~ - M2 F~) + M1 F~
    equals the weak-form DG residual with exact mass/stiffness/face integrals."""
    el = RefElement(etype, p)
    rng = np.random.default_rng(7)
    d, nu, nf = el.ndims, el.nupts, el.nfpts
    F = rng.standard_normal((d, nu))
    D = rng.standard_normal(nf)
    R_fr = el.M3 @ (D - el.M2 @ F.ravel()) + el.M1 @ F.ravel()
    ev = nodal_mono(el)
    Xq, Wq = vol_quad(etype, p + 4)
    Lq, dLq = ev(Xq)
    mass = (Lq * Wq) @ Lq.T
    Fq = F @ Lq                                       # [d, nq]
    rhs = -np.einsum("drq,dq,q->r", dLq, Fq, Wq)
    for X, W, Lf, ids in _face_rules(etype, el, p + 4):
        Lface, _ = ev(X)
        Dq = D[ids] @ Lf
        rhs += (Lface * W) @ Dq
    R_dg = np.linalg.solve(mass, rhs)
    assert np.allclose(R_fr, R_dg, atol=1e-11 * max(1.0, np.abs(R_dg).max()))


@pytest.mark.parametrize("etype,p", CASES)
def test_correction_integrates_to_face_weight(etype, p):
    """v = 1 in the lift definition: int(div g_sigma) = int_face l_sigma ds."""
    el = RefElement(etype, p)
    Xq, Wq = vol_quad(etype, p + 4)
    ev = nodal_mono(el)
    Lq, _ = ev(Xq)
    w_sol = Lq @ Wq
    lhs = w_sol @ el.M3
    rhs = np.zeros(el.nfpts)
    for X, W, Lf, ids in _face_rules(etype, el, p + 4):
        rhs[ids] = Lf @ W
    assert np.allclose(lhs, rhs, atol=1e-12)


def test_triangle_points_interior_and_unisolvent():
    for p in range(1, 7):
        el = RefElement("tri", p)
        x, y = el.upts.T
        assert np.all(x > -1) and np.all(y > -1) and np.all(x + y < 0)
        exps = monomial_exps("tri", p)
        Vm = mono(exps, el.upts.T)[0]
        assert np.linalg.matrix_rank(Vm) == len(exps)
