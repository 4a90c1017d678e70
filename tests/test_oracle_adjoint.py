"""Pins for the oracle's discrete adjoint (oracle/adjoint.py), Euler and
Navier-Stokes: the transpose is checked against the exact directional
derivative of the forward map taken by the complex-step method (an
independent route: the forward code in complex arithmetic), through the
dot-product identity <l, J v> = <J^T l, v>."""
import numpy as np
import pytest

from fr_inputs import periodic_box, annulus_mixed, fields
from fr_inputs.meshes import channel_mixed
from oracle.system import FRSystem
from oracle.adjoint import FRAdjoint, H_CS


NS_PRM = dict(mu=0.05, prandtl=0.72, ldg_beta=0.5, ldg_tau=0.1)


def _setup(kind, system="euler"):
    prm = dict(bc_rho=1.0, bc_v=(0.5, 0.1, 0.0), bc_p=2.0, outflow_p=2.0, wall_cpTw=3.5)
    if kind == "hex":
        m = periodic_box("hex", 2, 0.0, 2 * np.pi, jitter=0.1, seed=1)
        p = 3 if system == "euler" else 2
    elif kind == "channel":
        # isothermal walls at y = 0 and (moving) y = 1
        m = channel_mixed(3, 3, jitter=0.1, seed=5)
        p = 2
        prm.update(wall_v=(0.1, 0.0, 0.0), wall2_v=(0.7, -0.05, 0.0))
    else:
        m = annulus_mixed(ntheta=12, nr_quad=2, nr_tri=2, r0=0.5, r1=3.0, jitter=0.05, seed=3)
        m.bfaces[(m.bfaces[:, 0] == 1) & (m.bfaces[:, 1] % 2 == 0), 3] = 1     # some outflow faces
        p = 2
    if system == "ns":
        prm.update(NS_PRM)
    s = FRSystem(m, p, system, **prm)
    U = [fields.smooth_random(s.solution_coords(b), seed=2, amp=0.2, vel0=(0.5, 0.1, 0.0)[:m.ndims],
                              p0=2.0).transpose(1, 0, 2).copy() for b in range(len(s.eles))]
    return s, U


def _dot(a, b):
    return sum(float(np.sum(x * y)) for x, y in zip(a, b))


@pytest.mark.parametrize("kind,system", [("hex", "euler"), ("mixed", "euler"), ("hex", "ns"), ("mixed", "ns"),
                                         ("channel", "ns")])
def test_rhs_adjoint_dot_product(kind, system):
    s, U = _setup(kind, system)
    A = FRAdjoint(s)
    rng = np.random.default_rng(3)
    for _ in range(3):
        v = [rng.standard_normal(u.shape) for u in U]
        l = [rng.standard_normal(u.shape) for u in U]
        lhs, rhs = _dot(l, A.rhs_jvp(U, v)), _dot(A.rhs_vjp(U, l), v)
        assert abs(lhs - rhs) <= 1e-12 * abs(lhs)


def test_complex_step_jvp_matches_central_differences():
    """The complex-step JVP itself agrees with FP64 central differences."""
    s, U = _setup("hex")
    A = FRAdjoint(s)
    rng = np.random.default_rng(4)
    v = [rng.standard_normal(u.shape) for u in U]
    eps = 1e-6
    Rp = s.rhs([u + eps * dv for u, dv in zip(U, v)])
    Rm = s.rhs([u - eps * dv for u, dv in zip(U, v)])
    fd = [(a - b) / (2 * eps) for a, b in zip(Rp, Rm)]
    cs = A.rhs_jvp(U, v)
    assert np.allclose(fd[0], cs[0], rtol=1e-6, atol=1e-6 * np.abs(cs[0]).max())


def test_kinetic_energy_gradient():
    s, U = _setup("hex")
    A = FRAdjoint(s)
    rng = np.random.default_rng(5)
    v = [rng.standard_normal(u.shape) for u in U]
    cs = A.kinetic_energy([u + 1j * H_CS * dv for u, dv in zip(U, v)]).imag / H_CS
    assert abs(_dot(A.kinetic_energy_grad(U), v) - cs) <= 1e-12 * abs(cs)


@pytest.mark.parametrize("every,system", [(1, "euler"), (3, "euler"), (10, "euler"), (3, "ns")])
def test_rk4_adjoint_with_checkpoints(every, system):
    s, U = _setup("hex", system)
    A = FRAdjoint(s)
    dt, n = 2e-3, 7
    rng = np.random.default_rng(6)
    v = [rng.standard_normal(u.shape) for u in U]
    UN = s.rk4(U, dt, n)
    g = A.rk4_vjp(U, dt, n, A.kinetic_energy_grad(UN), every=every)
    Z = s.rk4([u + 1j * H_CS * dv for u, dv in zip(U, v)], dt, n)
    cs = A.kinetic_energy(Z).imag / H_CS
    assert abs(_dot(g, v) - cs) <= 1e-11 * abs(cs)


def test_ns_adjoint_differs_from_euler_adjoint():
    """The viscous terms reach the transpose: the NS adjoint at mu > 0 is not
    the Euler adjoint, and at mu = 0 with tau = 0 it is (same inviscid part)."""
    from oracle.system import FRSystem as S
    m = periodic_box("hex", 2, 0.0, 2 * np.pi, jitter=0.1, seed=1)
    e = S(m, 2, "euler")
    U = [fields.smooth_random(e.solution_coords(0), seed=2, amp=0.2, vel0=(0.5, 0.1, 0.0),
                              p0=2.0).transpose(1, 0, 2).copy()]
    lam = [np.random.default_rng(9).standard_normal(U[0].shape)]
    ge = FRAdjoint(e).rhs_vjp(U, lam)[0]
    g0 = FRAdjoint(S(m, 2, "ns", mu=0.0, ldg_tau=0.0)).rhs_vjp(U, lam)[0]
    g1 = FRAdjoint(S(m, 2, "ns", **NS_PRM)).rhs_vjp(U, lam)[0]
    assert np.abs(g0 - ge).max() <= 1e-12 * np.abs(ge).max()
    assert np.abs(g1 - ge).max() > 1e-3 * np.abs(ge).max()
