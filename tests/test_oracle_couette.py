"""Pins of the oracle on the Couette channel (Sec. 5.2): mixed quad/triangle
channel periodic in x with an isothermal wall at rest below and the second
(moving) isothermal wall type above."""

import numpy as np
import pytest

from fr_inputs import fields
from fr_inputs.meshes import channel_mixed
from oracle.system import FRSystem
from tests.libutil import oracle_state

G, PR, CPTW, VW, PC, MU = 1.4, 0.72, 1005.0 * 300.0, 69.445, 1e5, 0.417
PRM = dict(gamma=G, mu=MU, prandtl=PR, ldg_beta=0.5, ldg_tau=0.1, wall_cpTw=CPTW,
           wall_v=(0.0, 0.0, 0.0), wall2_v=(VW, 0.0, 0.0))


def test_channel_mesh_boundaries():
    m = channel_mixed(6, 4, jitter=0.1, seed=3)
    assert [b.etype for b in m.blocks] == ["quad", "tri"]
    o = FRSystem(m, 2, "ns", **PRM)                       # pairs every interior / periodic point
    # every boundary face lies on y = 0 (type 2) or y = 1 (type 3)
    for b, e, f, t in m.bfaces:
        el = o.eles[b]
        ids = el.face_fpts[f]
        yf = o.geo[b]["Xf"][e][ids, 1]
        assert np.allclose(yf, 0.0 if t == 2 else 1.0, atol=1e-14), (b, e, f, t)
    assert sorted(set(m.bfaces[:, 3].tolist())) == [2, 3]
    assert np.sum(m.bfaces[:, 3] == 2) == 6 and np.sum(m.bfaces[:, 3] == 3) == 6


def test_rest_state_at_wall_temperature_is_steady():
    m = channel_mixed(5, 5, jitter=0.1, seed=2)
    o = FRSystem(m, 3, "ns", **dict(PRM, wall2_v=(0.0, 0.0, 0.0)))
    rho0 = G / (G - 1) * PC / CPTW
    U = oracle_state(o, lambda X: fields.uniform(X, rho0, (0.0, 0.0), PC, G))
    R, S = o.rhs(U, scale=True)
    # at rest the density terms vanish; the pressure terms set the round-off scale
    smax = max(s.max() for s in S)
    for r in R:
        assert np.abs(r).max() <= 1e-13 * smax


def test_couette_mass_is_conserved():
    m = channel_mixed(5, 4, jitter=0.1, seed=4)
    o = FRSystem(m, 2, "ns", **PRM)
    U = oracle_state(o, lambda X: fields.couette(X, G, PR, CPTW, VW, PC))
    U = [u * (1 + 0.01 * np.sin(np.arange(u.size)).reshape(u.shape)) for u in U]   # off the steady state
    R = o.rhs(U)
    tot = sum(np.einsum("un,un->", o.quadrature_weights(b), R[b][:, 0]) for b in range(len(R)))
    scale = sum(np.einsum("un,un->", o.quadrature_weights(b), np.abs(R[b][:, 0])) for b in range(len(R)))
    assert abs(tot) < 1e-12 * scale


@pytest.mark.parametrize("p", [2, 3])
def test_exact_couette_state_residual_converges(p):
    # the analytic steady state is a steady state of the PDE: the semi-discrete
    # residual at it is the truncation error of the first derivatives, O(h^p)
    res = []
    for n in (4, 8, 16):
        m = channel_mixed(n, n, jitter=0.1, seed=1)
        o = FRSystem(m, p, "ns", **PRM)
        U = oracle_state(o, lambda X: fields.couette(X, G, PR, CPTW, VW, PC))
        res.append(max(np.abs(r[:, -1]).max() for r in o.rhs(U)))
    rates = np.log2(np.array(res[:-1]) / np.array(res[1:]))
    assert np.all(rates > p - 0.4), rates
