"""GPU discrete adjoint (fr_adjoint_rhs, fr_rk4_adjoint, FRStep), Euler and
Navier-Stokes, against the oracle's adjoint and against FP64 central finite
differences.

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
from oracle.adjoint import FRAdjoint
from tests.libutil import ensure_built, rel_l2_per_var

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch():
    import torch as t
    assert t.cuda.is_available()
    ensure_built()
    return t


NS_PRM = dict(mu=0.05, prandtl=0.72, ldg_beta=0.5, ldg_tau=0.1)


def _case(kind, system="euler"):
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
    if system == "ns":
        prm = dict(prm, **NS_PRM)
        p = min(p, 3)
    o = FRSystem(m, p, system, **prm)
    U = [fields.smooth_random(o.solution_coords(b), seed=2, amp=0.2, vel0=(0.5, 0.1, 0.0)[:m.ndims],
                              p0=2.0).transpose(1, 0, 2).copy() for b in range(len(o.eles))]
    return m, p, prm, o, U


# single precision: the Euler chain (one operator pair around the flux
# Jacobians) is held to rel-L2 2e-5; the Navier-Stokes chain adds the
# transposed gradient stage (M0^T, J^-1, M6^T and M4 - M6 M0 around the
# viscous-flux Jacobians), a second derivative-operator pair, hence 5e-5
@pytest.mark.parametrize("system", ["euler", "ns"])
@pytest.mark.parametrize("kind", ["hex", "mixed", "channel"])
@pytest.mark.parametrize("prec", ["fp64", "fp32", "tf32x3"])
def test_adjoint_rhs_matches_oracle(torch, kind, prec, system):
    from paper_1312_1638_b300 import fr
    tol = {"fp64": 1e-12, "fp32": 2e-5, "tf32x3": 2e-5}[prec] * (2.5 if system == "ns" and prec != "fp64" else 1)
    m, p, prm, o, U = _case(kind, system)
    if prec != "fp64":
        U = [u.astype(np.float32).astype(np.float64) for u in U]
    rng = np.random.default_rng(7)
    lam = [rng.standard_normal(u.shape) for u in U]
    if prec != "fp64":
        lam = [l.astype(np.float32).astype(np.float64) for l in lam]
    ref = FRAdjoint(o).rhs_vjp(U, lam)
    s = fr.Solver(m, p, system, prec, device=0, **prm)
    tu = [torch.from_numpy(s.pack(b, U[b])).cuda() for b in range(len(U))]
    tl = [torch.from_numpy(s.pack(b, lam[b])).cuda() for b in range(len(U))]
    to = [torch.zeros_like(x) for x in tu]
    s.adjoint_rhs(tu, tl, to)
    torch.cuda.synchronize()
    errs = []
    for b in range(len(U)):
        g = to[b].cpu().numpy()[:, :, :U[b].shape[2]].astype(np.float64)
        errs.append(rel_l2_per_var(g, ref[b]))
    print(f"adjoint {system} {kind} {prec}: rel-L2 {max(errs):.2e} (bound {tol:.0e})")
    assert max(errs) <= tol
    assert s.sync_status() == fr.OK


def test_ns_adjoint_repeatable_and_forward_unchanged(torch):
    """The NS adjoint reuses the forward scratch: repeated calls give the same
    bits, and an RHS evaluated afterwards equals one evaluated before."""
    from paper_1312_1638_b300 import fr
    m, p, prm, o, U = _case("mixed", "ns")
    s = fr.Solver(m, p, "ns", "fp64", device=0, **prm)
    tu = [torch.from_numpy(s.pack(b, U[b])).cuda() for b in range(len(U))]
    rng = np.random.default_rng(8)
    tl = [torch.from_numpy(s.pack(b, rng.standard_normal(U[b].shape))).cuda() for b in range(len(U))]
    r0 = [torch.zeros_like(x) for x in tu]
    s.rhs(tu, r0)
    outs = []
    for _ in range(2):
        to = [torch.zeros_like(x) for x in tu]
        s.adjoint_rhs(tu, tl, to)
        outs.append([x.clone() for x in to])
    r1 = [torch.zeros_like(x) for x in tu]
    s.rhs(tu, r1)
    torch.cuda.synchronize()
    for a, b in zip(*outs):
        assert torch.equal(a, b)
    for a, b in zip(r0, r1):
        assert torch.equal(a, b)


@pytest.mark.parametrize("system", ["euler", "ns"])
def test_rk4_adjoint_matches_oracle(torch, system):
    from paper_1312_1638_b300 import fr
    m = periodic_box("hex", 2, 0.0, 2 * np.pi, jitter=0.1, seed=1)
    prm = NS_PRM if system == "ns" else {}
    o = FRSystem(m, 3, system, **prm)
    A = FRAdjoint(o)
    U = [fields.smooth_random(o.solution_coords(0), seed=2, amp=0.2, vel0=(0.5, 0.1, 0.0),
                              p0=2.0).transpose(1, 0, 2).copy()]
    dt, n, every = 2e-3, 7, 3
    lamN = A.kinetic_energy_grad(o.rk4(U, dt, n))
    ref = A.rk4_vjp(U, dt, n, lamN, every=every)
    s = fr.Solver(m, 3, system, "fp64", device=0, **prm)
    u0 = torch.from_numpy(s.pack(0, U[0])).cuda()
    lam = torch.from_numpy(s.pack(0, lamN[0])).cuda()
    s.rk4_adjoint([u0], [lam], dt, n, every)
    g = lam.cpu().numpy()[:, :, :m.nelem]
    assert rel_l2_per_var(g, ref[0]) <= 1e-11
    assert np.array_equal(u0.cpu().numpy()[:, :, :m.nelem], U[0])     # u0 untouched


@pytest.mark.parametrize("system", ["euler", "ns"])
def test_autograd_gradcheck_tiny(torch, system):
    from paper_1312_1638_b300 import fr
    from paper_1312_1638_b300.autograd import FRStep
    m = periodic_box("hex", 1, 0.0, 1.0)
    s = fr.Solver(m, 1, system, "fp64", device=0, **(NS_PRM if system == "ns" else {}))
    X = s.solution_points(0)
    U = fields.smooth_random(X, period=1.0, seed=3, amp=0.1, vel0=(0.3, 0.0, 0.0)).transpose(1, 0, 2)
    lay = s.layout(0)
    x0 = torch.from_numpy(U.copy()).cuda().requires_grad_(True)            # the 40 real entries

    def f(x):
        u = torch.zeros((lay["nupts"], lay["nvars"], lay["ld"]), dtype=torch.float64, device="cuda")
        u = u.index_copy(2, torch.arange(m.nelem, device="cuda"), x)      # padded layout, differentiable
        return FRStep.apply(u, s, 1e-2, 2, 1)[:, :, :m.nelem]
    assert torch.autograd.gradcheck(f, (x0,), eps=1e-6, atol=1e-8, rtol=1e-6)


@pytest.mark.parametrize("prec", ["fp32", "tf32x3"])
def test_rk4_adjoint_against_fp64_finite_differences(torch, prec):
    """c4 in miniature: 3D Euler, periodic 4^3 hexes, p=4, Taylor-Green + seeded
    perturbation, 50 RK4 steps dt=1e-3, checkpoints every 10; gradient of the
    volume-integrated kinetic energy vs FP64 central differences on 200
    directions (tests/adjoint_fd_study.py)."""
    from tests.adjoint_fd_study import fd_check
    r = fd_check(4, 200, prec)
    assert not r["bad"], r["bad"][:5]


def test_rk4_adjoint_full_size_c4(torch):
    """c4 at full size (16^3 hexes, 2.56 M DOF), FP32 adjoint, 16 of the 200
    directions (the full set is the study's default run)."""
    from tests.adjoint_fd_study import fd_check
    r = fd_check(16, 16, "fp32")
    assert not r["bad"], r["bad"][:5]


def test_ns_rk4_adjoint_against_fp64_finite_differences(torch):
    """The c4 check on the Navier-Stokes equations: 3D NS (Taylor-Green
    constants), periodic 4^3 hexes, p=4, Taylor-Green + seeded perturbation,
    50 RK4 steps dt=1e-3, checkpoints every 10, FP32 adjoint in plain
    variables; 64 seeded directions against FP64 central differences."""
    from tests.adjoint_fd_study import fd_check
    r = fd_check(4, 64, "fp32", system="ns")
    assert not r["bad"], r["bad"][:5]


@pytest.mark.parametrize("system", ["euler", "ns"])
def test_autograd_gradcheck_mixed_mesh_blocks(torch, system):
    """FRStepBlocks on a two-block mesh (quadrilaterals with a curved wall ring
    and triangles, wall and free-stream boundaries): torch's gradcheck of the
    tuple of block states against central differences of fr_rk4."""
    from fr_inputs import annulus_mixed
    from paper_1312_1638_b300 import fr
    from paper_1312_1638_b300.autograd import rk4
    m = annulus_mixed(ntheta=6, nr_quad=1, nr_tri=1, r0=0.5, r1=2.0, jitter=0.05, seed=5)
    prm = dict(gamma=1.4, bc_rho=1.0, bc_v=(0.5, 0.1, 0.0), bc_p=2.0, outflow_p=2.0, wall_cpTw=3.5)
    if system == "ns":
        prm.update(NS_PRM)
    s = fr.Solver(m, 1, system, "fp64", device=0, **prm)
    xs, lays = [], []
    for b in range(s.nblocks):
        X = s.solution_points(b)
        U = fields.smooth_random(X, seed=3 + b, amp=0.05, vel0=(0.5, 0.1), p0=2.0).transpose(1, 0, 2)
        xs.append(torch.from_numpy(U.copy()).cuda().requires_grad_(True))
        lays.append(s.layout(b))

    def f(*x):
        u = []
        for b, (xb, lay) in enumerate(zip(x, lays)):
            ub = torch.zeros((lay["nupts"], lay["nvars"], lay["ld"]), dtype=torch.float64, device="cuda")
            u.append(ub.index_copy(2, torch.arange(lay["nelem"], device="cuda"), xb))
        out = rk4(s, u, 1e-3, 2, 1)
        return tuple(o[:, :, :lay["nelem"]] for o, lay in zip(out, lays))
    assert torch.autograd.gradcheck(f, tuple(xs), eps=1e-6, atol=1e-7, rtol=1e-6)
    assert s.sync_status() == fr.OK
