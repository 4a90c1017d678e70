"""GPU discrete adjoint (fr_adjoint_rhs, fr_rk4_adjoint, FRStep) against the
oracle's adjoint and against FP64 central finite differences.

Tolerances: FP64 rel-L2 <= 1e-12 against the oracle's transpose (both are
exact transposes of the same discretisation).  Single-precision adjoints are
checked on the gradient of the kinetic energy after 50 RK4 steps against FP64
central differences on 200 seeded directions with the criterion
|g.d - FD| <= 1e-4 (|FD| + 1e-3 |g| |d|).
"""
import ctypes as C

import numpy as np
import pytest

from fr_inputs import periodic_box, annulus_mixed, fields
from oracle.system import FRSystem
from oracle.adjoint import EulerAdjoint
from tests.libutil import ensure_built, rel_l2_per_var

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch():
    import torch as t
    assert t.cuda.is_available()
    ensure_built()
    return t


def _case(kind):
    if kind == "hex":
        m = periodic_box("hex", 3, 0.0, 2 * np.pi, jitter=0.1, seed=1)
        p, prm = 3, dict(gamma=1.4)
    elif kind == "channel":
        # walls at rest below and moving above (boundary types 2 and 3)
        from fr_inputs.meshes import channel_mixed
        m = channel_mixed(4, 4, jitter=0.1, seed=5)
        p, prm = 2, dict(gamma=1.4, wall_cpTw=3.5, wall_v=(0.1, 0.0, 0.0), wall2_v=(0.7, -0.05, 0.0))
    else:
        m = annulus_mixed(ntheta=16, nr_quad=2, nr_tri=2, r0=0.5, r1=3.0, jitter=0.05, seed=3)
        m.bfaces[(m.bfaces[:, 0] == 1) & (m.bfaces[:, 1] % 2 == 0), 3] = 1
        p, prm = 3, dict(gamma=1.4, bc_rho=1.0, bc_v=(0.5, 0.1, 0.0), bc_p=2.0, outflow_p=2.0, wall_cpTw=3.5)
    o = FRSystem(m, p, "euler", **prm)
    U = [fields.smooth_random(o.solution_coords(b), seed=2, amp=0.2, vel0=(0.5, 0.1, 0.0)[:m.ndims],
                              p0=2.0).transpose(1, 0, 2).copy() for b in range(len(o.eles))]
    return m, p, prm, o, U


@pytest.mark.parametrize("kind", ["hex", "mixed", "channel"])
@pytest.mark.parametrize("prec,tol", [("fp64", 1e-12), ("fp32", 2e-5), ("tf32x3", 2e-5)])
def test_adjoint_rhs_matches_oracle(torch, kind, prec, tol):
    from paper_1312_1638_b300 import fr
    m, p, prm, o, U = _case(kind)
    if prec != "fp64":
        U = [u.astype(np.float32).astype(np.float64) for u in U]
    rng = np.random.default_rng(7)
    lam = [rng.standard_normal(u.shape) for u in U]
    if prec != "fp64":
        lam = [l.astype(np.float32).astype(np.float64) for l in lam]
    ref = EulerAdjoint(o).rhs_vjp(U, lam)
    s = fr.Solver(m, p, "euler", prec, device=0, **prm)
    tu = [torch.from_numpy(s.pack(b, U[b])).cuda() for b in range(len(U))]
    tl = [torch.from_numpy(s.pack(b, lam[b])).cuda() for b in range(len(U))]
    to = [torch.zeros_like(x) for x in tu]
    s.adjoint_rhs(tu, tl, to)
    torch.cuda.synchronize()
    for b in range(len(U)):
        g = to[b].cpu().numpy()[:, :, :U[b].shape[2]].astype(np.float64)
        assert rel_l2_per_var(g, ref[b]) <= tol
    assert s.sync_status() == fr.OK


def test_rk4_adjoint_matches_oracle(torch):
    from paper_1312_1638_b300 import fr
    m = periodic_box("hex", 2, 0.0, 2 * np.pi, jitter=0.1, seed=1)
    o = FRSystem(m, 3, "euler")
    A = EulerAdjoint(o)
    U = [fields.smooth_random(o.solution_coords(0), seed=2, amp=0.2, vel0=(0.5, 0.1, 0.0),
                              p0=2.0).transpose(1, 0, 2).copy()]
    dt, n, every = 2e-3, 7, 3
    lamN = A.kinetic_energy_grad(o.rk4(U, dt, n))
    ref = A.rk4_vjp(U, dt, n, lamN, every=every)
    s = fr.Solver(m, 3, "euler", "fp64", device=0)
    u0 = torch.from_numpy(s.pack(0, U[0])).cuda()
    lam = torch.from_numpy(s.pack(0, lamN[0])).cuda()
    s.rk4_adjoint([u0], [lam], dt, n, every)
    g = lam.cpu().numpy()[:, :, :m.nelem]
    assert rel_l2_per_var(g, ref[0]) <= 1e-11
    assert np.array_equal(u0.cpu().numpy()[:, :, :m.nelem], U[0])     # u0 untouched


def test_autograd_gradcheck_tiny(torch):
    from paper_1312_1638_b300 import fr
    from paper_1312_1638_b300.autograd import FRStep
    m = periodic_box("hex", 1, 0.0, 1.0)
    s = fr.Solver(m, 1, "euler", "fp64", device=0)
    X = s.solution_points(0)
    U = fields.smooth_random(X, period=1.0, seed=3, amp=0.1, vel0=(0.3, 0.0, 0.0)).transpose(1, 0, 2)
    lay = s.layout(0)
    x0 = torch.from_numpy(U.copy()).cuda().requires_grad_(True)            # the 40 real entries

    def f(x):
        u = torch.zeros((lay["nupts"], lay["nvars"], lay["ld"]), dtype=torch.float64, device="cuda")
        u = u.index_copy(2, torch.arange(m.nelem, device="cuda"), x)      # padded layout, differentiable
        return FRStep.apply(u, s, 1e-2, 2, 1)[:, :, :m.nelem]
    assert torch.autograd.gradcheck(f, (x0,), eps=1e-6, atol=1e-8, rtol=1e-6)


def _kinetic_energy(w, u, nelem):
    u = u[:, :, :nelem]
    m2 = (u[:, 1:4] ** 2).sum(1)
    return float((w * 0.5 * m2 / u[:, 0]).sum())


def _kinetic_energy_grad(w, u, nelem):
    g = np.zeros_like(u)
    uu = u[:, :, :nelem]
    m2 = (uu[:, 1:4] ** 2).sum(1)
    g[:, 0, :nelem] = -0.5 * w * m2 / uu[:, 0] ** 2
    for i in range(3):
        g[:, 1 + i, :nelem] = w * uu[:, 1 + i] / uu[:, 0]
    return g


def _replicated(box, copies, L):
    """`copies` disjoint copies of a periodic box in one element block, spaced
    10 L apart along x; the box's own translations keep each copy periodic in
    itself, so one RHS evaluates `copies` independent states."""
    from fr_inputs import Mesh, Block
    nodes = box.blocks[0].nodes
    allnodes = np.concatenate([nodes + np.array([10.0 * L * c, 0.0, 0.0]) for c in range(copies)])
    return Mesh(3, [Block("hex", allnodes)], box.bfaces, box.periodic)


@pytest.mark.parametrize("prec", ["fp32", "tf32x3"])
def test_rk4_adjoint_against_fp64_finite_differences(torch, prec):
    """c4 in miniature: 3D Euler, periodic 4^3 hexes, p=4, Taylor-Green + seeded
    perturbation, 50 RK4 steps dt=1e-3, checkpoints every 10; gradient of the
    volume-integrated kinetic energy vs FP64 central differences on 200
    directions d ~ N(0, I) scaled per variable by its RMS (default_rng(4242)).
    The FP64 trajectories run 8 directions at a time on 8 disjoint copies of
    the box."""
    from paper_1312_1638_b300 import fr
    L = 2 * np.pi
    m = periodic_box("hex", 4, 0.0, L)
    o = FRSystem(m, 4, "euler")
    w = o.quadrature_weights(0)
    U = fields.perturbed_taylor_green(o.solution_coords(0), M=0.1).transpose(1, 0, 2).copy()
    U = U.astype(np.float32).astype(np.float64)
    n, dt, every, ndir, batch = 50, 1e-3, 10, 200, 8
    s1 = fr.Solver(m, 4, "euler", prec, device=0)
    ne = m.nelem
    u0 = torch.from_numpy(s1.pack(0, U)).cuda()
    uN = u0.clone()
    s1.rk4([uN], dt, n)
    lam = torch.from_numpy(_kinetic_energy_grad(w, uN.cpu().numpy().astype(np.float64), ne).astype(np.float32)).cuda()
    s1.rk4_adjoint([u0], [lam], dt, n, every)
    g = lam.cpu().numpy().astype(np.float64)[:, :, :ne]
    rng = np.random.default_rng(4242)
    rms = np.sqrt((U ** 2).mean(axis=(0, 2)))
    dirs = [rng.standard_normal(U.shape) * rms[None, :, None] for _ in range(ndir)]
    mr = _replicated(m, batch, L)
    s64 = fr.Solver(mr, 4, "euler", "fp64", device=0)
    bad = []
    for k0 in range(0, ndir, batch):
        ds = dirs[k0:k0 + batch]
        eps = [1e-6 * np.sqrt((U ** 2).mean()) / np.sqrt((d ** 2).mean()) for d in ds]
        res = []
        for sign in (1.0, -1.0):
            Ub = np.concatenate([U + sign * e * d for e, d in zip(eps, ds)], axis=2)
            ub = torch.from_numpy(s64.pack(0, Ub)).cuda()
            s64.rk4([ub], dt, n)
            uh = ub.cpu().numpy()
            res.append([_kinetic_energy(w, uh[:, :, c * ne:(c + 1) * ne], ne) for c in range(len(ds))])
        for c, (d, e) in enumerate(zip(ds, eps)):
            fd = (res[0][c] - res[1][c]) / (2 * e)
            gd = float(np.sum(g * d))
            if abs(gd - fd) > 1e-4 * (abs(fd) + 1e-3 * np.linalg.norm(g) * np.linalg.norm(d)):
                bad.append((k0 + c, gd, fd))
    assert not bad, bad[:5]
