"""Pins for the sign of the LDG penalty tau (Sec. 4.3).

As printed, the viscous common flux contains +tau (u_L - u_R) and the common
flux subtracts it, which would make the penalty anti-dissipative; the oracle
(and the library) read it as a dissipative penalty, F = ... + tau (u_L - u_R).
Two checks fix that sign independently of how the oracle spells it:

* Energy identity.  On an affine periodic mesh with Gauss-Legendre solution
  and flux points, solution-point quadrature is the exact mass matrix and the
  DG correction lifts face values with the exact face quadrature, so the
  penalty's contribution Delta R = R(tau) - R(0) produces
  sum_e sum_rho w_rho J_rho u . Delta R = -tau sum_pairs w_f |J n| |u_L - u_R|^2
  (w_f the face Gauss weight of the pair's flux point, |J n| its face
  Jacobian, the same on both sides of a conforming affine face): never
  positive, and zero only for a continuous trace.
* Energy decay.  A small-amplitude shear wave v = (0, eps sin x) with a
  temperature wave rho = 1 + eps sin y at uniform pressure is a steady state
  of the inviscid equations that viscosity and heat conduction damp; the
  discrete energy sum w J |u - u_mean|^2 under RK4 must not grow at any step
  for tau in {0, 0.1, 1, 3}, must end lower the larger tau is, and the printed
  sign (tau -> -tau) at tau = 3 must make it grow.
"""
import numpy as np
import pytest

from fr_inputs import periodic_box, fields
from oracle.polys import gauss_legendre
from oracle.system import FRSystem

L = 2 * np.pi
KW = dict(mu=0.05, prandtl=0.72)


def _state(s, fn):
    return [fn(s.solution_coords(b)).transpose(1, 0, 2).copy() for b in range(len(s.eles))]


@pytest.mark.parametrize("etype,n,p", [("quad", 3, 2), ("quad", 2, 3), ("hex", 2, 2)])
@pytest.mark.parametrize("tau", [0.1, 1.0])
def test_penalty_energy_identity(etype, n, p, tau):
    m = periodic_box(etype, n, 0.0, L)
    s0 = FRSystem(m, p, "ns", ldg_tau=0.0, **KW)
    st = FRSystem(m, p, "ns", ldg_tau=tau, **KW)
    rng = np.random.default_rng(7)
    U = _state(s0, lambda X: fields.smooth_random(X, period=L, seed=5, amp=0.2))
    U = [u + 1e-2 * rng.standard_normal(u.shape) for u in U]      # jumps at every face
    dR = st.rhs(U)[0] - s0.rhs(U)[0]
    w = s0.quadrature_weights(0)
    production = float(np.einsum("un,uvn,uvn->", w, U[0], dR))
    # right-hand side of the identity from the trace jumps
    el = s0.eles[0]
    Uf = np.einsum("fu,uvn->fvn", el.M0, U[0])
    P = s0.pairs
    jump2 = np.sum((Uf[P["fL"], :, P["nL"]] - Uf[P["fR"], :, P["nR"]]) ** 2, axis=1)
    _, w1 = gauss_legendre(p + 1)
    wf = w1 if etype == "quad" else np.outer(w1, w1).ravel()
    assert np.allclose(P["magL"], P["magR"], rtol=1e-13)
    expected = -tau * float(np.sum(wf[P["fL"] % len(wf)] * P["magL"] * jump2))
    assert expected < 0.0
    assert production < 0.0
    assert abs(production - expected) <= 1e-10 * abs(expected)


def _shear_temperature_wave(X, eps=1e-3):
    x, y = X[0], X[1]
    return fields.conserved(1.0 + eps * np.sin(y), (0.0 * x, eps * np.sin(x)), np.ones_like(x), 1.4)


def _energy_history(tau, nsteps=60, dt=5e-3):
    m = periodic_box("quad", 4, 0.0, L)
    s = FRSystem(m, 2, "ns", ldg_tau=tau, **KW)
    U = _state(s, _shear_temperature_wave)
    w = s.quadrature_weights(0)
    ubar = np.einsum("un,uvn->v", w, U[0]) / w.sum()

    def energy(U):
        d = U[0] - ubar[None, :, None]
        return float(np.einsum("un,uvn->", w, d * d))

    E = [energy(U)]
    for _ in range(nsteps):
        U = s.rk4(U, dt, 1)
        E.append(energy(U))
    return np.array(E)


def test_penalty_energy_decay_and_printed_sign_growth():
    hist = {tau: _energy_history(tau) for tau in (0.0, 0.1, 1.0, 3.0)}
    for tau, E in hist.items():
        assert np.all(np.diff(E) <= 0.0), tau                     # no step adds energy
        assert E[-1] < E[0], tau
    ends = [hist[t][-1] for t in (0.0, 0.1, 1.0, 3.0)]
    assert all(a > b for a, b in zip(ends, ends[1:]))             # a larger penalty damps more
    printed = _energy_history(-3.0)                               # the sign as printed, tau = 3
    assert printed[-1] > 10.0 * printed[0]
