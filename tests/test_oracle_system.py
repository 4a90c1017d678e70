"""Pins for the assembled oracle RHS: pairing invariants (Sec. 2), freestream
preservation, discrete conservation (Eq. commpflux), RK4 amplification, p+1
convergence on the isentropic vortex (Sec. 5.1) and convergence of the
Navier-Stokes RHS to the PDE differentiated symbolically (Sec. 4)."""
import numpy as np
import pytest
import sympy as sp

from fr_inputs import periodic_box, annulus_mixed, fields
from oracle.system import FRSystem
from oracle.geometry import map_points


def state(sysm, fn):
    return [fn(sysm.solution_coords(b)).transpose(1, 0, 2).copy() for b in range(len(sysm.eles))]


@pytest.mark.parametrize("etype,n,p", [("quad", 3, 2), ("hex", 2, 2)])
def test_pairs_coincide_with_opposite_normals(etype, n, p):
    m = periodic_box(etype, n, 0.0, 1.0, jitter=0.1, seed=2)
    s = FRSystem(m, p)
    P = s.pairs
    L = 2 * np.pi
    for k in range(len(P["bL"])):
        gL, gR = s.geo[P["bL"][k]], s.geo[P["bR"][k]]
        xl, xr = gL["Xf"][P["nL"][k], P["fL"][k]], gR["Xf"][P["nR"][k], P["fR"][k]]
        dx = xl - xr
        assert np.allclose(dx - np.round(dx), 0.0, atol=1e-12)       # periodic images on [0,1]
        assert np.allclose(gL["nrm"][P["nL"][k], P["fL"][k]], -gR["nrm"][P["nR"][k], P["fR"][k]], atol=1e-12)
    # every flux point belongs to exactly one pair
    el = s.eles[0]
    seen = np.zeros((m.nelem, el.nfpts), int)
    np.add.at(seen, (P["nL"], P["fL"]), 1)
    np.add.at(seen, (P["nR"], P["fR"]), 1)
    assert np.all(seen == 1)
    del L


FS = dict(rho=1.3, v=(0.3, -0.2, 0.1), p=2.0)


def uniform_fn(nd):
    return lambda X: fields.uniform(X, FS["rho"], FS["v"][:nd], FS["p"], 1.4)


@pytest.mark.parametrize("system", ["euler", "ns"])
@pytest.mark.parametrize("etype,n,p,jit", [("quad", 3, 1, 0.0), ("quad", 4, 3, 0.15),
                                           ("hex", 2, 2, 0.0), ("hex", 2, 2, 0.15), ("hex", 2, 3, 0.1)])
def test_freestream_preserved_periodic(system, etype, n, p, jit):
    m = periodic_box(etype, n, 0.0, 2.0, jitter=jit, seed=11)
    s = FRSystem(m, p, system, mu=0.02)
    R = s.rhs(state(s, uniform_fn(m.ndims)))
    assert np.abs(R[0]).max() < 1e-12


@pytest.mark.parametrize("system", ["euler", "ns"])
def test_freestream_preserved_curved_mixed_with_boundaries(system):
    m = annulus_mixed(ntheta=16, nr_quad=2, nr_tri=2, r0=0.5, r1=3.0, jitter=0.05, seed=3)
    m.bfaces[:, 3] = 0                    # every boundary free-stream at the same state
    s = FRSystem(m, 3, system, mu=0.02, bc_rho=FS["rho"], bc_v=FS["v"], bc_p=FS["p"])
    R = s.rhs(state(s, uniform_fn(2)))
    for r in R:
        assert np.abs(r).max() < 1e-11


@pytest.mark.parametrize("system", ["euler", "ns"])
@pytest.mark.parametrize("etype,n,p", [("quad", 4, 3), ("hex", 2, 2)])
def test_discrete_conservation_periodic(system, etype, n, p):
    L = 2 * np.pi
    m = periodic_box(etype, n, 0.0, L, jitter=0.12, seed=4)
    s = FRSystem(m, p, system, mu=0.05)
    U = state(s, lambda X: fields.smooth_random(X, period=L, seed=9, amp=0.2))
    R = s.rhs(U)
    w = s.quadrature_weights(0)
    tot = np.einsum("un,uvn->v", w, R[0])
    scale = np.einsum("un,uvn->v", w, np.abs(R[0]))
    assert np.all(np.abs(tot) < 1e-12 * scale.max())


def test_conservation_mixed_mesh_wall_has_no_mass_flux():
    """Mass is conserved up to the free-stream boundary flux; with all
    boundaries walls the total mass change is zero (no-slip ghost carries
    no mass through the Rusanov flux when v_L=0 at the wall)."""
    m = annulus_mixed(ntheta=12, nr_quad=2, nr_tri=1, r0=0.5, r1=2.0, jitter=0.0, seed=3)
    m.bfaces[:, 3] = 2
    s = FRSystem(m, 2, "ns", mu=0.02, wall_cpTw=3.5)
    U = state(s, lambda X: fields.uniform(X, 1.0, (0.0, 0.0), 1.0, 1.4))
    R = s.rhs(U)
    tot = sum(np.einsum("un,un->", s.quadrature_weights(b), R[b][:, 0]) for b in range(2))
    assert abs(tot) < 1e-12


def test_rk4_amplification_factor():
    m = periodic_box("quad", 2, 0.0, 1.0)
    s = FRSystem(m, 1)
    lam = -0.7 + 0.4j
    s.rhs = lambda U: [lam * u for u in U]
    U = [np.ones((4, 4, 4), complex)]
    for z in (0.1, 0.5, 1.3):
        out = s.rk4(U, z / lam, 1)[0]
        zz = z
        expect = 1 + zz + zz ** 2 / 2 + zz ** 3 / 6 + zz ** 4 / 24
        assert np.allclose(out, expect, rtol=1e-14)


def _vortex_error(n, p, tend=0.5, cfl=0.02, correction="dg"):
    m = periodic_box("quad", n, -10.0, 10.0)
    s = FRSystem(m, p, "euler", gamma=1.4, correction=correction)
    U = state(s, lambda X: fields.isentropic_vortex(X, S=5.0, M=0.4, R=1.5))
    h = 20.0 / n
    nst = int(np.ceil(tend / (cfl * h)))
    U = s.rk4(U, tend / nst, nst)
    el = s.eles[0]
    xq, wq = np.polynomial.legendre.leggauss(p + 3)
    XQ = np.array([(a, b) for b in xq for a in xq]).T
    WQ = np.array([wa * wb for wb in wq for wa in wq])
    Xq, J = map_points("quad", m.blocks[0].nodes, XQ)
    rho = np.einsum("uq,un->nq", el.nodal(XQ), U[0][:, 0, :])
    ex = fields.isentropic_vortex(Xq.transpose(2, 0, 1), S=5.0, M=0.4, R=1.5, t=tend)[0]
    return np.sqrt(np.sum((rho - ex) ** 2 * np.linalg.det(J) * WQ))


@pytest.mark.parametrize("p", [2, 3])
def test_isentropic_vortex_order_p_plus_one(p):
    ns = [14, 20, 28]
    errs = [_vortex_error(n, p) for n in ns]
    slope = np.polyfit(np.log(20.0 / np.array(ns)), np.log(errs), 1)[0]
    assert slope > p + 1 - 0.4, (errs, slope)


def _ns_exact_rhs_2d(mu, Pr, gam):
    x, y = sp.symbols("x y")
    g = sp.nsimplify(gam)
    Cv = 1
    Cp = g * Cv
    rho = 1 + sp.Rational(1, 5) * sp.sin(x) * sp.cos(y)
    vx = sp.Rational(3, 10) + sp.Rational(1, 10) * sp.sin(y)
    vy = sp.Rational(1, 10) * sp.cos(x + y)
    p = 1 + sp.Rational(1, 10) * sp.cos(x)
    E = p / (g - 1) + rho * (vx ** 2 + vy ** 2) / 2
    v, X = [vx, vy], [x, y]
    T = p / (rho * Cv * (g - 1))
    div = sum(sp.diff(v[i], X[i]) for i in range(2))
    tau = [[mu * (sp.diff(v[j], X[i]) + sp.diff(v[i], X[j])) - (sp.Rational(2, 3) * mu * div if i == j else 0)
            for j in range(2)] for i in range(2)]
    Delta = mu * Cp / Pr
    u = [rho, rho * vx, rho * vy, E]
    finv = [[rho * v[i], rho * vx * v[i] + (p if i == 0 else 0), rho * vy * v[i] + (p if i == 1 else 0),
             v[i] * (E + p)] for i in range(2)]
    fvis = [[0, tau[0][i], tau[1][i], sum(v[j] * tau[j][i] for j in range(2)) + Delta * sp.diff(T, X[i])]
            for i in range(2)]
    R = [-(sum(sp.diff(finv[i][a] - fvis[i][a], X[i]) for i in range(2))) for a in range(4)]
    return sp.lambdify((x, y), u, "numpy"), sp.lambdify((x, y), R, "numpy")


@pytest.mark.parametrize("system,p,min_rate", [("euler", 3, 2.6), ("ns", 3, 1.7)])
def test_rhs_converges_to_symbolic_pde(system, p, min_rate):
    mu = 0.05 if system == "ns" else 0.0
    fu, fR = _ns_exact_rhs_2d(sp.Rational(1, 20) if system == "ns" else 0, sp.Rational(18, 25), 1.4)
    errs = []
    for n in (4, 8, 16):
        m = periodic_box("quad", n, 0.0, 2 * np.pi, jitter=0.1, seed=5)
        s = FRSystem(m, p, system, gamma=1.4, mu=mu, prandtl=0.72)
        X = s.solution_coords(0)
        U = np.array([np.broadcast_to(a, X[0].shape) for a in fu(X[0], X[1])])
        Rex = np.array([np.broadcast_to(a, X[0].shape) for a in fR(X[0], X[1])])
        Rd = s.rhs([U.transpose(1, 0, 2).copy()])[0].transpose(1, 0, 2)
        w = s.quadrature_weights(0)
        errs.append(np.sqrt(np.sum(w * (Rd - Rex) ** 2, axis=(1, 2))))
    errs = np.array(errs)
    rates = np.log2(errs[:-1] / errs[1:])
    assert np.all(rates[-1] > min_rate), rates
