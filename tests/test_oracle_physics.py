"""Pins for oracle.physics and oracle.geometry: properties that fix the Euler
flux (hyperbolic eigenstructure), the Rusanov solver (consistency,
conservation, wave speed = spectral radius), LDG limits, ghost states (read
back through the ideal-gas inversion) and the metric terms (finite differences,
edge lengths)."""
import numpy as np
import pytest

from oracle import physics as ph
from oracle.geometry import map_points, flux_point_metrics, solution_point_metrics
from oracle.elements import RefElement

G = 1.4


def rand_state(nd, rng, n=5):
    rho = rng.uniform(0.5, 2.0, n)
    v = rng.uniform(-1, 1, (nd, n))
    p = rng.uniform(0.5, 3.0, n)
    E = p / (G - 1) + 0.5 * rho * (v * v).sum(0)
    return np.vstack([rho, rho * v, E])


def unit(nd, rng, n=5):
    v = rng.standard_normal((nd, n))
    return v / np.linalg.norm(v, axis=0)


def cs_jacobian(fun, u, h=1e-30):
    """Complex-step Jacobian of fun: R^V -> R^V at a single state u[V]."""
    V = len(u)
    J = np.empty((V, V))
    for k in range(V):
        du = np.zeros(V, complex); du[k] = 1j * h
        J[:, k] = fun(u + du).imag / h
    return J


@pytest.mark.parametrize("nd", [2, 3])
def test_euler_flux_eigenvalues(nd):
    rng = np.random.default_rng(1)
    u = rand_state(nd, rng, 1)[:, 0]
    n = unit(nd, rng, 1)[:, 0]
    fun = lambda w: np.einsum("i,iv->v", n, ph.inviscid_flux(w[:, None], G)[:, :, 0])
    J = cs_jacobian(fun, u.astype(complex))
    rho, v, p = u[0], u[1:1 + nd] / u[0], None
    p = (G - 1) * (u[-1] - 0.5 * rho * v @ v)
    c = np.sqrt(G * p / rho)
    vn = v @ n
    lam = np.sort(np.linalg.eigvals(J).real)
    expect = np.sort([vn - c] + [vn] * nd + [vn + c])
    assert np.allclose(lam, expect, atol=1e-10)


@pytest.mark.parametrize("nd", [2, 3])
def test_euler_flux_homogeneous_degree_one(nd):
    rng = np.random.default_rng(2)
    u = rand_state(nd, rng)
    assert np.allclose(ph.inviscid_flux(3.7 * u, G), 3.7 * ph.inviscid_flux(u, G), rtol=1e-13)


@pytest.mark.parametrize("nd", [2, 3])
def test_rusanov_consistency_conservation_wavespeed(nd):
    rng = np.random.default_rng(3)
    uL, uR = rand_state(nd, rng), rand_state(nd, rng)
    n = unit(nd, rng)
    f = ph.inviscid_flux(uL, G)
    assert np.allclose(ph.rusanov(uL, uL, n, G), np.einsum("in,ivn->vn", n, f), rtol=1e-13, atol=1e-13)
    assert np.allclose(ph.rusanov(uL, uR, n, G), -ph.rusanov(uR, uL, -n, G), rtol=1e-13, atol=1e-13)
    # dissipation coefficient -> spectral radius of n.df/du as u_R -> u_L
    u = uL[:, 0]
    nn = n[:, 0]
    eps = 1e-7
    du = rng.standard_normal(len(u)) * eps
    F = ph.rusanov((u + du)[:, None], u[:, None], nn[:, None], G)[:, 0]
    cen = 0.5 * np.einsum("i,iv->v", nn, ph.inviscid_flux((u + du)[:, None], G)[:, :, 0]
                          + ph.inviscid_flux(u[:, None], G)[:, :, 0])
    s = ((F - cen) / (0.5 * du)).mean()
    fun = lambda w: np.einsum("i,iv->v", nn, ph.inviscid_flux(w[:, None], G)[:, :, 0])
    J = cs_jacobian(fun, u.astype(complex))
    assert abs(s - np.abs(np.linalg.eigvals(J)).max()) < 1e-6


def test_ldg_common_solution_limits():
    rng = np.random.default_rng(4)
    uL, uR = rand_state(2, rng), rand_state(2, rng)
    assert np.allclose(ph.ldg_common_solution(uL, uL, 0.3), uL)
    assert np.allclose(ph.ldg_common_solution(uL, uR, 0.5), uR)
    assert np.allclose(ph.ldg_common_solution(uL, uR, -0.5), uL)


@pytest.mark.parametrize("nd", [2, 3])
def test_viscous_flux_linear_in_gradient_and_zero_for_uniform(nd):
    rng = np.random.default_rng(5)
    u = rand_state(nd, rng)
    q1, q2 = rng.standard_normal((2, nd, nd + 2, 5))
    f = lambda q: ph.viscous_flux(u, q, G, 0.3, 0.72)
    assert np.allclose(f(2 * q1 - 0.5 * q2), 2 * f(q1) - 0.5 * f(q2), atol=1e-12)
    assert np.allclose(f(np.zeros_like(q1)), 0.0)
    # the mass row carries no viscous flux
    assert np.allclose(f(q1)[:, 0], 0.0)


def test_viscous_stress_traceless_in_3d():
    rng = np.random.default_rng(6)
    u = rand_state(3, rng)
    q = rng.standard_normal((3, 5, 5))
    f = ph.viscous_flux(u, q, G, 0.3, 0.72)
    # f[i, 1+j] = T_ij; in 3D the Stokes stress is traceless
    assert np.allclose(f[0, 1] + f[1, 2] + f[2, 3], 0.0, atol=1e-12)
    assert np.allclose(f[0, 2], f[1, 1]) and np.allclose(f[0, 3], f[2, 1])


def test_ghost_states_read_back():
    rng = np.random.default_rng(7)
    uL = rand_state(2, rng)
    prm = dict(gamma=G, bc_rho=1.2, bc_v=(0.4, -0.1, 0.0), bc_p=2.5, outflow_p=1.7,
               wall_cpTw=3.0, wall_v=(0.2, 0.0, 0.0))
    gi, gl, _ = ph.ghost_states(ph.BC_INFLOW, uL, None, prm)
    rho, v, p = ph.primitives(gi, G)
    assert np.allclose(rho, 1.2) and np.allclose(v[0], 0.4) and np.allclose(v[1], -0.1) and np.allclose(p, 2.5)
    assert np.array_equal(gi, gl)
    gi, gl, _ = ph.ghost_states(ph.BC_OUTFLOW, uL, None, prm)
    rho, v, p = ph.primitives(gi, G)
    r0, v0, _ = ph.primitives(uL, G)
    assert np.allclose(rho, r0) and np.allclose(v[0], v0[0]) and np.allclose(p, 1.7)
    q = rng.standard_normal((2, 4, 5))
    gi, gl, qg = ph.ghost_states(ph.BC_WALL, uL, q, prm)
    ri, vi, pi = ph.primitives(gi, G)
    rl, vl, pl = ph.primitives(gl, G)
    # mirrored velocity averages to the wall velocity; LDG ghost moves with the wall
    assert np.allclose(0.5 * (vi[0] + v0[0]), 0.2) and np.allclose(0.5 * (vi[1] + v0[1]), 0.0)
    assert np.allclose(vl[0], 0.2) and np.allclose(vl[1], 0.0)
    # both ghosts sit at the wall temperature: C_p T = gamma/(gamma-1) p/rho
    assert np.allclose(G / (G - 1) * pi / ri, 3.0) and np.allclose(G / (G - 1) * pl / rl, 3.0)
    assert np.array_equal(qg, q)
    # the second wall type moves at wall2_v at the same temperature
    prm2 = dict(prm, wall2_v=(-0.5, 0.3, 0.0))
    gi, gl, qg = ph.ghost_states(ph.BC_WALL2, uL, q, prm2)
    ri, vi, pi = ph.primitives(gi, G)
    rl, vl, pl = ph.primitives(gl, G)
    assert np.allclose(0.5 * (vi[0] + v0[0]), -0.5) and np.allclose(0.5 * (vi[1] + v0[1]), 0.3)
    assert np.allclose(vl[0], -0.5) and np.allclose(vl[1], 0.3)
    assert np.allclose(G / (G - 1) * pl / rl, 3.0) and np.array_equal(qg, q)


@pytest.mark.parametrize("etype,nn", [("quad", 4), ("quad", 9), ("tri", 3), ("tri", 6), ("hex", 8)])
def test_jacobian_matches_finite_differences(etype, nn):
    rng = np.random.default_rng(8)
    el = RefElement(etype, 2)
    ref = {"quad": 4, "tri": 3, "hex": 8}[etype]
    # a valid element: perturbed standard element (curved for 9/6 nodes)
    from oracle.geometry import shape_functions
    nodes_std = {"quad": [(-1, -1), (1, -1), (-1, 1), (1, 1)], "tri": [(-1, -1), (1, -1), (-1, 1)],
                 "hex": [(a, b, c) for c in (-1, 1) for b in (-1, 1) for a in (-1, 1)]}[etype]
    std = np.array(nodes_std, float)
    if nn == 9:
        std = np.array([(a, b) for b in (-1, 0, 1) for a in (-1, 0, 1)], float)
    if nn == 6:
        std = np.vstack([std, [(0, -1), (0, 0), (-1, 0)]])
    nodes = (std + 0.1 * rng.standard_normal(std.shape))[None]
    x = el.upts.T
    X, J = map_points(etype, nodes, x)
    h = 1e-6
    for j in range(el.ndims):
        dx = np.zeros_like(x); dx[j] = h
        Xp, _ = map_points(etype, nodes, x + dx)
        Xm, _ = map_points(etype, nodes, x - dx)
        assert np.allclose((Xp - Xm) / (2 * h), J[..., :, j], atol=1e-8)
    # partition of unity of the shape functions
    N, dN = shape_functions(etype, nodes.shape[1], x)
    assert np.allclose(N.sum(0), 1.0) and np.allclose(dN.sum(1), 0.0, atol=1e-13)
    del ref


def test_face_metrics_integrate_to_edge_lengths():
    rng = np.random.default_rng(9)
    el = RefElement("quad", 3)
    std = np.array([(-1, -1), (1, -1), (-1, 1), (1, 1)], float)
    nodes = (std * 1.7 + 0.2 * rng.standard_normal(std.shape))[None]
    Xf, mag, nrm, _ = flux_point_metrics("quad", nodes, el.fpts, el.fnorm)
    w = np.polynomial.legendre.leggauss(4)[1]
    edges = [(0, 1), (1, 3), (3, 2), (2, 0)]
    for f, (a, b) in enumerate(edges):
        ids = el.face_fpts[f]
        length = np.linalg.norm(nodes[0, b] - nodes[0, a])
        assert np.isclose((w * mag[0, ids]).sum(), length, rtol=1e-13)
        t = (nodes[0, b] - nodes[0, a]) / length
        outward = np.array([t[1], -t[0]])                   # CCW boundary: normal = tangent rotated -90
        assert np.allclose(nrm[0, ids], outward, atol=1e-13)
    _, det, adj = solution_point_metrics("quad", nodes, el.upts)
    assert np.all(det > 0)


def test_affine_hex_metrics_closed_form():
    A = np.array([[1.3, 0.2, 0.0], [0.1, 0.9, 0.3], [0.0, -0.2, 1.1]])
    c = np.array([0.5, -1.0, 2.0])
    std = np.array([(a, b, cc) for cc in (-1, 1) for b in (-1, 1) for a in (-1, 1)], float)
    nodes = (std @ A.T + c)[None]
    el = RefElement("hex", 2)
    X, det, adj = solution_point_metrics("hex", nodes, el.upts)
    assert np.allclose(det, np.linalg.det(A))
    assert np.allclose(adj, np.linalg.det(A) * np.linalg.inv(A))
    assert np.allclose(X[0], el.upts @ A.T + c)
